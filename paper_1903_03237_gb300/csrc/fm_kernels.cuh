// FastMNMF kernels, templated on MAXM (the channel bucket: 2, 4 or 8).  Included by
// fm_kernels_m{2,4,8}.cu, each of which instantiates one bucket.
//
// One iteration (Sec. III, block order W -> H -> g~ -> Q -> normalise) is six launches:
//   k_tile<MODE_W>   W update, Eq. 23:   num/den[n,k,f] = sum_t h_nkt sum_m g~_nfm {x~/y~^2, 1/y~}
//   k_tile<MODE_H>   H update, Eq. 24:   num/den[n,k,t] = sum_f w_nkf sum_m g~_nfm {x~/y~^2, 1/y~}
//   k_tile<MODE_G>   g~ update, Eq. 21:  num/den[n,f,m] = sum_t lambda_ftn {x~/y~^2, 1/y~}
//   k_tile<MODE_Y>   y~ refresh; split sums of V_fm = (1/T) sum_t x x^H / y~_ftm (Eq. 18)
//   k_ip             IP, Eqs. 19-20, float-float, one CTA per bin (+ phi and nu normalisation)
//   k_xt_ll          x~ = |Q_f x_ft|^2 (below Eq. 17); log-likelihood, Eq. 17; mu normalisation
// A k_tile CTA owns kOT consecutive "own" elements and one split of the summed "inner"
// index; each split writes partial sums and the last CTA to arrive for an own tile sums
// the splits in a fixed order and applies the update, so results do not depend on
// scheduling.  lambda_ftn = sum_k w_nkf h_nkt (Eq. 9) is formed on chip from W and H
// tiles staged in shared memory; it is never written to memory.
#pragma once
#include "fm_common.cuh"
#include "fm_df64.cuh"

namespace fm {

enum { MODE_W = 0, MODE_H = 1, MODE_G = 2, MODE_Y = 3 };
// FLAG_DO_V (MODE_Y): form V_fm and run the IP update.  FLAG_UPDATE (MODE_G): apply the
// g~ rule (without it the launch only normalises).  FLAG_NORMALISE: scale normalisation.
// FLAG_LAM_MEM (MODE_G / MODE_Y): lambda is read from p.lam (mixed form) and the shared
// memory holds no factor tiles; the host sizes the launch's shared memory the same way.
enum { FLAG_DO_V = 1, FLAG_NORMALISE = 2, FLAG_UPDATE = 4, FLAG_LAM_MEM = 8 };

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float dot4acc(float4 a, float4 b, float c) {
  c = fmaf(a.x, b.x, c); c = fmaf(a.y, b.y, c); c = fmaf(a.z, b.z, c); return fmaf(a.w, b.w, c);
}
__device__ __forceinline__ bool finitef(float v) { return isfinite(v); }

// Shared-memory carve-up of k_tile (in floats; every region a multiple of 4 floats).
// "o" is the own index within the tile (kOT), "i" the inner index within the sub-chunk
// (IC, rows padded to ICP = IC + 4 so that 16-byte rows fall on different banks).
struct TileSmem {
  int own, oth, gw, gi, xs, ys, xc, a, b, acc, total;
};
__host__ __device__ inline int r4(int x) { return (x + 3) & ~3; }
// lam_mem: lambda is read from memory (mixed form, MODE_G / MODE_Y): no factor tiles.
__host__ __device__ inline TileSmem tile_smem(int mode, int N, int K, int M, int MAXM, int IC, bool lam_mem = false) {
  const int ICP = IC + 4, NK = N * K;
  const bool f_own = (mode != MODE_H);
  TileSmem s;
  int o = 0;
  s.own = o; o += (mode != MODE_W && !lam_mem) ? NK * kOT : 0;  // own factor tile [NK][kOT]
  s.oth = o; o += lam_mem ? 0 : NK * ICP;                        // other factor chunk [NK][ICP]
  s.gw = o;  o += f_own ? r4(N * kOT * M) : 0;                // g~ of the own bins [N][kOT][M]
  s.gi = o;  o += (mode == MODE_H) ? N * M * ICP : 0;         // g~ of the chunk bins [N][M][ICP]
  s.xs = o;  o += (mode != MODE_Y) ? kOT * M * ICP : 0;       // x~ [kOT][M][ICP]
  s.ys = o;  o += (mode == MODE_W) ? kOT * M * ICP : 0;       // y~ [kOT][M][ICP]
  s.xc = o;  o += (mode == MODE_Y) ? r4(kOT * IC * M * 2) : 0;  // X [kOT][IC][M] complex
  s.a = o;
  if (mode == MODE_W || mode == MODE_H) o += 2 * N * kOT * ICP;  // P, R [2][N][kOT][ICP]
  if (mode == MODE_G) o += N * kOT * ICP;                        // lambda [N][kOT][ICP]
  s.b = o;
  if (mode == MODE_G) o += 2 * kOT * M * ICP;                    // A, B [2][kOT][M][ICP]
  if (mode == MODE_Y) o += kOT * M * ICP;                        // 1/y~ [kOT][M][ICP]
  s.acc = o;
  int accsz = (mode == MODE_W || mode == MODE_H) ? 2 * NK * kOT
            : (mode == MODE_G) ? 2 * N * kOT * M : kOT * M * MAXM * MAXM;
  o += r4(accsz);
  s.total = o;
  return s;
}

// 4- and 8-byte asynchronous global->shared copies (cp.async, L1-allocating); a copy with
// valid == false writes zeros and reads nothing.
__device__ __forceinline__ void cpa4(float* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cpa8(float2* dst, const float2* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cpa_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Sum of S split partials at p + ss*stride (ss = 0..S-1), in that order; loads issued
// eight at a time (predicated) so that their latencies overlap.
__device__ __forceinline__ float sum_splits(const float* p, size_t stride, int S) {
  float acc = 0.f;
  for (int ss = 0; ss < S; ss += 8) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = (ss + u < S) ? __ldcg(p + (size_t)(ss + u) * stride) : 0.f;
#pragma unroll
    for (int u = 0; u < 8; ++u) acc += v[u];
  }
  return acc;
}

// Partial-sum floats per split for each mode.
__host__ __device__ inline size_t tile_part_floats(int mode, int F, int T, int M, int N, int K, int MAXM) {
  switch (mode) {
    case MODE_W: return (size_t)2 * N * K * F;
    case MODE_H: return (size_t)2 * N * K * T;
    case MODE_G: return (size_t)2 * N * F * M;
    default: return (size_t)F * M * MAXM * MAXM;
  }
}

// 16-byte asynchronous copy (both addresses 16-byte aligned).
__device__ __forceinline__ void cpa16(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

// ---------------------------------------------------------------------------------
// Warp-level float64 linear algebra for the IP step (M <= 8).  A is row-major with
// leading dimension LD; columns [0, M) hold the matrix, columns [M, M + R) right-hand
// sides.  Gauss-Jordan with partial pivoting; returns false (all lanes) if a pivot is
// below 1e-30 times the largest entry of the matrix.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ double2 crecip(double2 b) {
  const double d = 1.0 / cabs2(b);
  return make_double2(b.x * d, -b.y * d);
}

// Lane-parallel partial pivot: the row r in [c, M) with the largest |A[r][c]|^2 (lowest
// row on ties), identical in every lane.
__device__ __forceinline__ int warp_pivot(int M, int LD, const double2* A, int c, double* best_out) {
  const int lane = threadIdx.x & 31;
  double v = (lane >= c && lane < M) ? cabs2(A[lane * LD + c]) : -1.0;
  int idx = lane;
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  *best_out = v;
  return idx;
}

__device__ inline bool warp_gauss_jordan(int M, int R, int LD, double2* A, double2* fac) {
  const int lane = threadIdx.x & 31;
  // scale for the singularity test
  double amax = 0.0;
  for (int e = lane; e < M * M; e += 32) amax = fmax(amax, cabs2(A[(e / M) * LD + (e % M)]));
  for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  bool ok = amax > 0.0 && isfinite(amax);
  const int C = M + R;
  for (int c = 0; c < M; ++c) {
    double bv;
    const int pr = warp_pivot(M, LD, A, c, &bv);
    ok = ok && (bv > 1e-60 * amax);
    if (pr != c) {
      for (int j = lane; j < C; j += 32) {
        double2 t = A[c * LD + j];
        A[c * LD + j] = A[pr * LD + j];
        A[pr * LD + j] = t;
      }
    }
    __syncwarp();
    const double2 inv = crecip(A[c * LD + c]);
    if (lane < M) fac[lane] = (lane == c) ? make_double2(0.0, 0.0) : cmul(A[lane * LD + c], inv);
    __syncwarp();
    for (int e = lane; e < M * C; e += 32) {
      int r = e / C, j = e % C;
      if (r != c && j >= c) A[r * LD + j] = csub(A[r * LD + j], cmul(fac[r], A[c * LD + j]));
    }
    __syncwarp();
  }
  // divide each row by its pivot
  for (int e = lane; e < M * R; e += 32) {
    int r = e / R, j = M + e % R;
    A[r * LD + j] = cmul(A[r * LD + j], crecip(A[r * LD + r]));
  }
  __syncwarp();
  return ok;
}

// log|det A|^2 by Gaussian elimination with partial pivoting (A is destroyed).
__device__ inline double warp_logdet2(int M, int LD, double2* A, double2* fac) {
  const int lane = threadIdx.x & 31;
  double prod = 1.0;  // product of |pivot|^2, renormalised by powers of two
  int ex = 0;
  for (int c = 0; c < M; ++c) {
    double bv;
    const int pr = warp_pivot(M, LD, A, c, &bv);
    if (pr != c) {
      for (int j = lane; j < M; j += 32) {
        double2 t = A[c * LD + j];
        A[c * LD + j] = A[pr * LD + j];
        A[pr * LD + j] = t;
      }
    }
    __syncwarp();
    const double2 pv = A[c * LD + c];
    int e2;
    prod = frexp(prod * cabs2(pv), &e2);
    ex += e2;
    const double2 inv = crecip(pv);
    if (lane < M) fac[lane] = (lane > c) ? cmul(A[lane * LD + c], inv) : make_double2(0.0, 0.0);
    __syncwarp();
    for (int e = lane; e < M * M; e += 32) {
      int r = e / M, j = e % M;
      if (r > c && j >= c) A[r * LD + j] = csub(A[r * LD + j], cmul(fac[r], A[c * LD + j]));
    }
    __syncwarp();
  }
  return log(prod) + (double)ex * 0.69314718055994531;  // log 2
}

// V_fm entry (j, c) from the packed Hermitian sums: slot a*MAXM+b holds Re(V_ab) for
// a <= b and Im(V_ba) for a > b.
template <int MAXM>
__device__ __forceinline__ double2 vget(const double* vs, int j, int c) {
  if (j == c) return make_double2(vs[j * MAXM + j], 0.0);
  if (j < c) return make_double2(vs[j * MAXM + c], vs[c * MAXM + j]);
  return make_double2(vs[c * MAXM + j], -vs[j * MAXM + c]);
}

// IP update of one bin by one warp, float64 (Eqs. 18-20), rows in order m = 0..M-1:
//   q <- (Q V_m)^-1 e_m ;  q <- q / sqrt(q^H V_m q) ;  row m of Q <- q^H
// vs: [M][MAXM*MAXM] packed V_fm (already divided by T).  Q: [MAXM*MAXM] in/out.
template <int MAXM>
__device__ bool warp_ip_bin(int M, const double* vs, double2* Q, double2* A, double2* fac, double2* qv) {
  const int lane = threadIdx.x & 31;
  const int LD = MAXM + 1;
  bool ok = true;
  for (int m = 0; m < M; ++m) {
    const double* v = vs + m * MAXM * MAXM;
    for (int e = lane; e < M * M; e += 32) {
      int r = e / M, c = e % M;
      double2 s = make_double2(0.0, 0.0);
      for (int j = 0; j < M; ++j) s = cadd(s, cmul(Q[r * MAXM + j], vget<MAXM>(v, j, c)));
      A[r * LD + c] = s;
    }
    if (lane < M) A[lane * LD + M] = make_double2(lane == m ? 1.0 : 0.0, 0.0);
    __syncwarp();
    ok = warp_gauss_jordan(M, 1, LD, A, fac) && ok;
    if (lane < M) qv[lane] = A[lane * LD + M];
    __syncwarp();
    // s = Re(q^H V q)
    double s = 0.0;
    for (int e = lane; e < M * M; e += 32) {
      int i = e / M, j = e % M;
      double2 t = cmul(cconj(qv[i]), cmul(vget<MAXM>(v, i, j), qv[j]));
      s += t.x;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (!(s > 0.0) || !isfinite(s)) { ok = false; s = 1.0; }
    const double inv = 1.0 / sqrt(s);
    if (lane < M) Q[m * MAXM + lane] = make_double2(qv[lane].x * inv, -qv[lane].y * inv);
    __syncwarp();
  }
  return ok;
}

// ---------------------------------------------------------------------------------
// The tiled sweep.  grid = (n_own_tiles, S), block = 256, dynamic smem = tile_smem(...).
// Per sub-chunk of the inner index: every operand the chunk needs is staged with
// cp.async (all copies in flight at once), then
//   phase 1: per point (2 own x 4 inner per item): lambda (unless MODE_W reads y~), y~,
//            and the ratios the mode needs;
//   phase 2: the contraction over the inner index into per-CTA accumulators.
// ---------------------------------------------------------------------------------
template <int MAXM, int MODE>
__global__ void __launch_bounds__(kThreads) k_tile(Prob p, Geom g, int flags, unsigned ctr_base) {
  extern __shared__ __align__(16) float sm[];
  constexpr bool F_OWN = (MODE != MODE_H);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = p.N, K = p.K, M = p.M, NK = N * K, F = p.F, T = p.T;
  const int SO = F_OWN ? F : T;
  const int SI = F_OWN ? T : F;
  const int ot = blockIdx.x, s = blockIdx.y;
  const int o_base = ot * kOT;
  const int n_own = min(kOT, SO - o_base);
  const int i_begin = s * g.span;
  const int i_end = min(SI, i_begin + g.span);
  const int IC = g.IC, ICP = g.ICP;
  const bool lam_mem = (MODE == MODE_G || MODE == MODE_Y) && (flags & FLAG_LAM_MEM);
  const TileSmem L = tile_smem(MODE, N, K, M, MAXM, IC, lam_mem);
  float* own_s = sm + L.own;
  float* oth_s = sm + L.oth;
  float* gw_s = sm + L.gw;
  float* gi_s = sm + L.gi;
  float* xs_s = sm + L.xs;
  float* ys_s = sm + L.ys;
  float2* xc_s = reinterpret_cast<float2*>(sm + L.xc);
  float* a_s = sm + L.a;
  float* b_s = sm + L.b;
  float* acc_s = sm + L.acc;

  const float* ownF = F_OWN ? p.W : p.H;
  const float* othF = F_OWN ? p.H : p.W;
  // mixed form (lam_mem): lambda was formed by the tensor-core GEMM and is read, not recomputed

  // once per CTA: own factor tile, g~ of the own bins, zeroed accumulators
  if (MODE != MODE_W && !lam_mem)
    for (int e = tid; e < NK * kOT; e += kThreads) {
      const int nk = e / kOT, o = e % kOT;
      cpa4(own_s + e, ownF + (size_t)nk * SO + o_base + min(o, n_own - 1), o < n_own);
    }
  if (F_OWN)
    for (int e = tid; e < N * kOT * M; e += kThreads) {
      const int n = e / (kOT * M), r = e % (kOT * M), o = r / M;
      cpa4(gw_s + e, p.G + ((size_t)n * F + o_base + min(o, n_own - 1)) * M + r % M, o < n_own);
    }
  {
    const int accsz = (MODE == MODE_W || MODE == MODE_H) ? 2 * NK * kOT
                    : (MODE == MODE_G) ? 2 * N * kOT * M : kOT * M * MAXM * MAXM;
    for (int e = tid; e < accsz; e += kThreads) acc_s[e] = 0.f;
  }

  const bool do_v = (MODE == MODE_Y) && (flags & FLAG_DO_V);
  for (int i0 = i_begin; i0 < i_end; i0 += IC) {
    const int icn = min(IC, i_end - i0);
    __syncthreads();  // previous sub-chunk fully consumed
    // ---- stage the chunk (asynchronous copies, zero-filled past its end) ----
    if (lam_mem) {
      // the other factor is not needed: lambda is read below
    } else if ((SI & 3) == 0 && (icn & 3) == 0) {
      // rows 16-byte aligned (SI, i0, IC multiples of 4): one 16-byte copy per 4 floats
      const int q = IC >> 2, qn = icn >> 2;
      for (int row = warp; row < NK; row += kThreads / 32) {
        const float* src = othF + (size_t)row * SI + i0;
        float* dst = oth_s + row * ICP;
        for (int j = lane; j < q; j += 32) {
          if (j < qn) cpa16(dst + 4 * j, src + 4 * j);
          else st4(dst + 4 * j, make_float4(0.f, 0.f, 0.f, 0.f));
        }
      }
    } else {
      for (int row = warp; row < NK; row += kThreads / 32) {
        const float* src = othF + (size_t)row * SI + i0;
        for (int i = lane; i < IC; i += 32) cpa4(oth_s + row * ICP + i, src + min(i, icn - 1), i < icn);
      }
    }
    if (MODE == MODE_W || MODE == MODE_G) {
      // x~ (and y~) of the own bins over the chunk frames, as [o][m][i]: one warp per
      // (o, m) row, lanes along the frames
      for (int row = warp; row < kOT * M; row += kThreads / 32) {
        const int o = row / M, m = row - o * M;
        const bool vo = o < n_own;
        const size_t base = ((size_t)(o_base + min(o, n_own - 1)) * T + i0) * M + m;
        float* dx = xs_s + row * ICP;
        float* dy = ys_s + row * ICP;
        for (int i = lane; i < IC; i += 32) {
          const bool v = vo && (i < icn);
          const size_t src = base + (size_t)min(i, icn - 1) * M;
          cpa4(dx + i, p.xt + src, v);
          if (MODE == MODE_W) cpa4(dy + i, p.yt + src, v);
        }
      }
    }
    if (MODE == MODE_H) {
      // x~ of the chunk bins over the own frames as [o][m][i]: for one bin the kOT*M values
      // of the own frames are contiguous; lanes along them, warps along the bins
      const int rowlen = kOT * M;
      for (int i = warp; i < IC; i += kThreads / 32) {
        const bool vi = i < icn;
        const size_t base = ((size_t)(i0 + min(i, icn - 1)) * T + o_base) * M;
        const int lim = n_own * M;
        for (int j = lane; j < rowlen; j += 32) cpa4(xs_s + j * ICP + i, p.xt + base + min(j, lim - 1), vi && j < lim);
      }
      // g~ of the chunk bins as [n][m][i]
      for (int row = warp; row < N * M; row += kThreads / 32) {
        const int n = row / M, m = row - n * M;
        const float* src = p.G + ((size_t)n * F + i0) * M + m;
        float* dst = gi_s + row * ICP;
        for (int i = lane; i < IC; i += 32) cpa4(dst + i, src + (size_t)min(i, icn - 1) * M, i < icn);
      }
    }
    if (do_v) {
      // X of the own bins over the chunk frames, [o][i][m] (the global layout): one warp per bin
      const int len = IC * M, lim = icn * M;
      for (int o = warp; o < kOT; o += kThreads / 32) {
        const bool vo = o < n_own;
        const float2* src = p.X + ((size_t)(o_base + min(o, n_own - 1)) * T + i0) * M;
        float2* dst = xc_s + o * len;
        for (int j = lane; j < len; j += 32) cpa8(dst + j, src + min(j, lim - 1), vo && j < lim);
      }
    }
    cpa_wait_all();
    __syncthreads();

    // ---------------- phase 1: per point quantities (2 own x 4 inner per item) -------
    const int nq = IC / 4;
    for (int it = tid; it < (kOT / 2) * nq; it += kThreads) {
      const int o0 = (it / nq) * 2;
      const int ii = (it % nq) * 4;
      float y[2][4][MAXM];
      if (MODE == MODE_W) {
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int m = 0; m < MAXM; ++m) {
            const float4 v = (m < M) ? ld4(ys_s + ((o0 + a) * M + m) * ICP + ii) : make_float4(1.f, 1.f, 1.f, 1.f);
            y[a][0][m] = v.x; y[a][1][m] = v.y; y[a][2][m] = v.z; y[a][3][m] = v.w;
          }
      } else {
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int m = 0; m < MAXM; ++m) y[a][b][m] = 0.f;
        for (int n = 0; n < N; ++n) {
          float lam[2][4];
#pragma unroll
          for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) lam[a][b] = 0.f;
          const float* ow = own_s + n * K * kOT + o0;
          const float* oh = oth_s + n * K * ICP + ii;
          if (lam_mem) {
#pragma unroll
            for (int a = 0; a < 2; ++a) {
              const int f = min(o_base + o0 + a, F - 1);
              const float* lp = p.lam + ((size_t)n * F + f) * T + i0 + ii;
#pragma unroll
              for (int b = 0; b < 4; ++b) lam[a][b] = (ii + b < icn) ? __ldg(lp + b) : 0.f;
            }
          }
#pragma unroll 4
          for (int k = 0; !lam_mem && k < K; ++k) {
            const float2 w = *reinterpret_cast<const float2*>(ow + k * kOT);
            const float4 h = ld4(oh + k * ICP);
            lam[0][0] = fmaf(w.x, h.x, lam[0][0]); lam[0][1] = fmaf(w.x, h.y, lam[0][1]);
            lam[0][2] = fmaf(w.x, h.z, lam[0][2]); lam[0][3] = fmaf(w.x, h.w, lam[0][3]);
            lam[1][0] = fmaf(w.y, h.x, lam[1][0]); lam[1][1] = fmaf(w.y, h.y, lam[1][1]);
            lam[1][2] = fmaf(w.y, h.z, lam[1][2]); lam[1][3] = fmaf(w.y, h.w, lam[1][3]);
          }
          if (MODE == MODE_G) {
            st4(a_s + (n * kOT + o0) * ICP + ii, make_float4(lam[0][0], lam[0][1], lam[0][2], lam[0][3]));
            st4(a_s + (n * kOT + o0 + 1) * ICP + ii, make_float4(lam[1][0], lam[1][1], lam[1][2], lam[1][3]));
          }
#pragma unroll
          for (int m = 0; m < MAXM; ++m) {
            if (m < M) {
              if (F_OWN) {
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                  const float gv = gw_s[(n * kOT + o0 + a) * M + m];
#pragma unroll
                  for (int b = 0; b < 4; ++b) y[a][b][m] = fmaf(lam[a][b], gv, y[a][b][m]);
                }
              } else {
                const float4 gv = ld4(gi_s + (n * M + m) * ICP + ii);
                const float gg[4] = {gv.x, gv.y, gv.z, gv.w};
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                  for (int b = 0; b < 4; ++b) y[a][b][m] = fmaf(lam[a][b], gg[b], y[a][b][m]);
              }
            }
          }
        }
      }

      if (MODE == MODE_Y) {
        // write y~ (before the phi normalisation) and 1/y~
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          float binv[4][MAXM];
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const bool v = (o0 + a < n_own) && (ii + b < icn);
            const size_t pt = (size_t)(o_base + o0 + a) * T + (i0 + ii + b);
#pragma unroll
            for (int m = 0; m < MAXM; ++m) {
              binv[b][m] = 0.f;
              if (v && m < M) {
                p.yt[pt * M + m] = y[a][b][m];
                binv[b][m] = __fdividef(1.f, y[a][b][m]);
              }
            }
          }
          if (do_v) {
#pragma unroll
            for (int m = 0; m < MAXM; ++m)
              if (m < M) st4(b_s + ((o0 + a) * M + m) * ICP + ii, make_float4(binv[0][m], binv[1][m], binv[2][m], binv[3][m]));
          }
        }
      } else {
        // A = x~ / y~^2, B = 1 / y~ (zero outside the chunk / tile)
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          float A[4][MAXM], B[4][MAXM];
#pragma unroll
          for (int m = 0; m < MAXM; ++m) {
            const float4 xv = (m < M) ? ld4(xs_s + ((o0 + a) * M + m) * ICP + ii) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float xx[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              const bool v = (o0 + a < n_own) && (ii + b < icn) && (m < M);
              const float bi = v ? __fdividef(1.f, y[a][b][m]) : 0.f;
              B[b][m] = bi;
              A[b][m] = xx[b] * bi * bi;
            }
          }
          if (MODE == MODE_G) {
#pragma unroll
            for (int m = 0; m < MAXM; ++m)
              if (m < M) {
                st4(b_s + ((0 * kOT + o0 + a) * M + m) * ICP + ii, make_float4(A[0][m], A[1][m], A[2][m], A[3][m]));
                st4(b_s + ((1 * kOT + o0 + a) * M + m) * ICP + ii, make_float4(B[0][m], B[1][m], B[2][m], B[3][m]));
              }
          } else {
            // P_n = sum_m g~ A,  R_n = sum_m g~ B
            for (int n = 0; n < N; ++n) {
              float P4[4] = {0.f, 0.f, 0.f, 0.f}, R4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
              for (int m = 0; m < MAXM; ++m)
                if (m < M) {
                  if (F_OWN) {
                    const float gv = gw_s[(n * kOT + o0 + a) * M + m];
#pragma unroll
                    for (int b = 0; b < 4; ++b) { P4[b] = fmaf(gv, A[b][m], P4[b]); R4[b] = fmaf(gv, B[b][m], R4[b]); }
                  } else {
                    const float4 gv = ld4(gi_s + (n * M + m) * ICP + ii);
                    const float gg[4] = {gv.x, gv.y, gv.z, gv.w};
#pragma unroll
                    for (int b = 0; b < 4; ++b) { P4[b] = fmaf(gg[b], A[b][m], P4[b]); R4[b] = fmaf(gg[b], B[b][m], R4[b]); }
                  }
                }
              st4(a_s + ((0 * N + n) * kOT + o0 + a) * ICP + ii, make_float4(P4[0], P4[1], P4[2], P4[3]));
              st4(a_s + ((1 * N + n) * kOT + o0 + a) * ICP + ii, make_float4(R4[0], R4[1], R4[2], R4[3]));
            }
          }
        }
      }
    }
    __syncthreads();

    // ---------------- phase 2: contraction over the inner index ----------------------
    const int icn4 = (icn + 3) & ~3;
    if (MODE == MODE_W || MODE == MODE_H) {
      const int KP = (K + 1) >> 1;
      const int ntl = N * KP * (kOT / 2);
      for (int tl = tid; tl < ntl; tl += kThreads) {
        const int o0 = (tl & 3) * 2;
        const int kp = (tl >> 2) % KP;
        const int n = (tl >> 2) / KP;
        const int k0 = 2 * kp;
        const bool has1 = (k0 + 1 < K);
        const int k1 = has1 ? k0 + 1 : k0;
        const float* P0 = a_s + ((0 * N + n) * kOT + o0) * ICP;
        const float* P1 = P0 + ICP;
        const float* R0 = a_s + ((1 * N + n) * kOT + o0) * ICP;
        const float* R1 = R0 + ICP;
        const float* h0 = oth_s + (n * K + k0) * ICP;
        const float* h1 = oth_s + (n * K + k1) * ICP;
        float c[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
        for (int i = 0; i < icn4; i += 4) {
          const float4 p0 = ld4(P0 + i), p1 = ld4(P1 + i), r0 = ld4(R0 + i), r1 = ld4(R1 + i);
          const float4 x0 = ld4(h0 + i), x1 = ld4(h1 + i);
          c[0] = dot4acc(x0, p0, c[0]); c[1] = dot4acc(x0, p1, c[1]);
          c[2] = dot4acc(x1, p0, c[2]); c[3] = dot4acc(x1, p1, c[3]);
          c[4] = dot4acc(x0, r0, c[4]); c[5] = dot4acc(x0, r1, c[5]);
          c[6] = dot4acc(x1, r0, c[6]); c[7] = dot4acc(x1, r1, c[7]);
        }
        float* an = acc_s + (0 * NK + n * K + k0) * kOT + o0;
        float* ad = acc_s + (1 * NK + n * K + k0) * kOT + o0;
        an[0] += c[0]; an[1] += c[1]; ad[0] += c[4]; ad[1] += c[5];
        if (has1) { an[kOT] += c[2]; an[kOT + 1] += c[3]; ad[kOT] += c[6]; ad[kOT + 1] += c[7]; }
      }
    } else if (MODE == MODE_G) {
      const int ntl = N * kOT * M;
      for (int tl = tid; tl < ntl; tl += kThreads) {
        const int m = tl % M, o = (tl / M) % kOT, n = tl / (M * kOT);
        const float* lp = a_s + (n * kOT + o) * ICP;
        const float* ap = b_s + ((0 * kOT + o) * M + m) * ICP;
        const float* bp = b_s + ((1 * kOT + o) * M + m) * ICP;
        float cn = 0.f, cd = 0.f;
        for (int i = 0; i < icn4; i += 4) {
          const float4 l = ld4(lp + i);
          cn = dot4acc(l, ld4(ap + i), cn);
          cd = dot4acc(l, ld4(bp + i), cd);
        }
        acc_s[((0 * N + n) * kOT + o) * M + m] += cn;
        acc_s[((1 * N + n) * kOT + o) * M + m] += cd;
      }
    } else if (do_v) {
      // V_fm partial sums: warp w <-> own bin o = w; lane = (m, t-subset), IS = 32 / MP
      // lanes per channel (MP = MAXM rounded to a power of two), MAXM^2 accumulators each
      constexpr int MM = MAXM * MAXM;
      constexpr int IS = 32 / MAXM;
      const int o = warp;
      const int m = lane / IS, isub = lane % IS;
      float acc[MM];
#pragma unroll
      for (int q = 0; q < MM; ++q) acc[q] = 0.f;
      if (o < n_own && m < M) {
        const float* bp = b_s + (o * M + m) * ICP;
        for (int i = isub; i < icn; i += IS) {
          const float2* xp = xc_s + (o * IC + i) * M;
          float2 x[MAXM];
#pragma unroll
          for (int j = 0; j < MAXM; ++j) x[j] = (j < M) ? xp[j] : make_float2(0.f, 0.f);
          const float bv = bp[i];
#pragma unroll
          for (int a = 0; a < MAXM; ++a)
#pragma unroll
            for (int c = 0; c < MAXM; ++c) {
              const float pr = (a <= c) ? (x[a].x * x[c].x + x[a].y * x[c].y)     // Re(x_a conj x_c)
                                        : (x[c].y * x[a].x - x[c].x * x[a].y);    // Im(x_c conj x_a)
              acc[a * MAXM + c] = fmaf(bv, pr, acc[a * MAXM + c]);
            }
        }
      }
#pragma unroll
      for (int q = 0; q < MM; ++q) {
        float v = acc[q];
#pragma unroll
        for (int off = IS >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        acc[q] = v;
      }
      if (o < n_own && m < M && isub == 0) {
#pragma unroll
        for (int q = 0; q < MM; ++q) acc_s[(o * M + m) * MM + q] += acc[q];
      }
    }
  }
  __syncthreads();

  // ---------------- write this split's partial sums ---------------------------------
  if (MODE == MODE_Y && !do_v) return;
  const size_t psz = tile_part_floats(MODE, F, T, M, N, K, MAXM);
  float* part = p.part + (size_t)s * psz;
  if (MODE == MODE_W || MODE == MODE_H) {
    for (int e = tid; e < 2 * NK * kOT; e += kThreads) {
      const int o = e % kOT, r = e / kOT;  // r = pr*NK + nk
      if (o < n_own) part[(size_t)r * SO + o_base + o] = acc_s[e];
    }
  } else if (MODE == MODE_G) {
    for (int e = tid; e < 2 * N * kOT * M; e += kThreads) {
      const int m = e % M, o = (e / M) % kOT, r = e / (M * kOT);  // r = pr*N + n
      if (o < n_own) part[((size_t)r * F + o_base + o) * M + m] = acc_s[e];
    }
  } else {
    constexpr int MM = MAXM * MAXM;
    for (int e = tid; e < kOT * M * MM; e += kThreads) {
      const int o = e / (M * MM);
      if (o < n_own) part[(size_t)(o_base)*M * MM + e] = acc_s[e];
    }
    return;  // k_ip reduces the V_fm splits
  }
  // Every split must have finished reading the state before the last one rewrites it.
  if (!arrive_last(p.counters + ctr_base + ot, g.S)) return;

  // ---------------- last CTA of this own tile: reduce splits, apply the update -------
  if (MODE == MODE_W || MODE == MODE_H) {
    float* __restrict__ fac = F_OWN ? p.W : p.H;
    const float* __restrict__ pp = p.part;
    for (int e0 = 0; e0 < NK * kOT; e0 += 4 * kThreads) {
      float ratio[4], old[4];
      size_t idx[4];
      bool ok[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + u * kThreads + tid;
        const int nk = e / kOT, o = e % kOT;
        ok[u] = (e < NK * kOT) && (o < n_own);
        idx[u] = ok[u] ? (size_t)nk * SO + o_base + o : 0;
        const float num = ok[u] ? sum_splits(pp + idx[u], psz, g.S) : 1.f;
        const float den = ok[u] ? sum_splits(pp + (size_t)NK * SO + idx[u], psz, g.S) : 1.f;
        ratio[u] = num / den;
        old[u] = ok[u] ? fac[idx[u]] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (ok[u]) {
          const float v = old[u] * sqrtf(ratio[u]);
          if (!finitef(v)) flag(p.status, ST_NONFINITE);
          fac[idx[u]] = v;
        }
    }
  } else {
    // g~ <- g~ sqrt(num/den)
    for (int e = tid; e < N * kOT * M; e += kThreads) {
      const int m = e % M, o = (e / M) % kOT, n = e / (M * kOT);
      if (o >= n_own) continue;
      const size_t idx = ((size_t)n * F + o_base + o) * M + m;
      const float num = sum_splits(p.part + idx, psz, g.S);
      const float den = sum_splits(p.part + (size_t)N * F * M + idx, psz, g.S);
      const float v = p.G[idx] * sqrtf(num / den);
      if (!finitef(v)) flag(p.status, ST_NONFINITE);
      p.G[idx] = v;
    }
  }
}

// ---------------------------------------------------------------------------------
// IP update (Eqs. 18-20) and the per-bin normalisation.  One CTA per bin, float-float
// arithmetic (about 48 significand bits) on the FP32 pipes.
//
// Eq. 19 solves (Q_f V_fm) q = e_m with the current Q_f.  Since (Q_f V_fm)^-1 =
// V_fm^-1 Q_f^-1, q = V_fm^-1 c_m with c_m = Q_f^-1 e_m.  V_fm depends only on y~, so the
// M inverses are formed first, in parallel (warp m sweeps V_fm: Hermitian positive
// definite, no pivoting).  Warp 0 then runs the rows in order m = 0..M-1 (ip_rows, with
// Q_f^-1 in registers):
//   q = V_fm^-1 c_m,   s = c_m^H q  (= q^H V_fm q, Eq. 20),   q_new = q / sqrt(s),
//   row m of Q_f <- q_new^H,
//   Q_f^-1 <- Q_f^-1 - c_m (q_new^H Q_f^-1 - e_m^T) / sqrt(s)   (Sherman-Morrison),
//   log|det Q_f|^2 += log s                                      (determinant lemma),
// so Q_f^-1 and log|det Q_f|^2 are carried across iterations instead of re-factored.
// Then phi_f = tr(Q_f Q_f^H)/M: Q_f /= sqrt(phi), Q_f^-1 *= sqrt(phi), g~_nf /= phi,
// log|det|^2 -= M log phi; nu_nf = sum_m g~_nfm: g~_nf /= nu, w_nkf *= nu.
// With xt_mode the same CTA then computes x~ = |Q_f x_ft|^2 for its bin's frames with the
// new Q_f (y~ /= phi_f) and the bin's log-likelihood terms; the bins are added up in bin
// order (Eq. 17) by the last CTA to finish or by a later kernel (ll_tail).
// ---------------------------------------------------------------------------------
// P_n = sum_m g~_nfm x~_m / y~_m^2 and R_n = sum_m g~_nfm / y~_m at one TF point (the
// per-point factors of the W and H updates, Eqs. 23-24), into PR[n][pt] and PR[N + n][pt]
// (source stride ns).  g points at g~_{0f0}, source stride gs.  Every kernel that forms
// them calls this one definition, so they all produce the same bits.
template <int MAXM>
__device__ __forceinline__ void pr_point(const float (&x)[MAXM], const float (&y)[MAXM], int M, int N,
                                         const float* g, size_t gs, float* PR, size_t ns, size_t pt) {
  float A[MAXM], B[MAXM];
#pragma unroll
  for (int m = 0; m < MAXM; ++m) {
    B[m] = (m < M) ? __fdividef(1.f, y[m]) : 0.f;
    A[m] = x[m] * B[m] * B[m];
  }
  for (int n = 0; n < N; ++n) {
    const float* gn = g + (size_t)n * gs;
    float P = 0.f, R = 0.f;
#pragma unroll
    for (int m = 0; m < MAXM; ++m)
      if (m < M) { P = fmaf(gn[m], A[m], P); R = fmaf(gn[m], B[m], R); }
    PR[(size_t)n * ns + pt] = P;
    PR[(size_t)(N + n) * ns + pt] = R;
  }
}

// In-place Gauss-Jordan inverse of one Hermitian positive definite V_fm on one warp, in
// float-float, with the matrix in registers: lane l holds entries (i, j), j = l % MAXM,
// i = l / MAXM + r * IG (the layout of ip_rows).  v holds the packed split sums (real parts
// on and above the diagonal, imaginary parts below); the inverse goes to A (row-major,
// leading dimension MAXM).  Per pivot k the pivot row and column come by shuffles:
//   A[k][k] <- 1/p,  A[k][j] <- A[k][j]/p,  A[i][k] <- -A[i][k]/p,
//   A[i][j] <- A[i][j] - A[i][k] (A[k][j]/p)          (p = A[k][k], no pivoting).
// Returns false (on every lane) when a pivot is not positive and finite.
// vlo (may be null): low parts of the sums, when they were accumulated in float-float.
template <int MAXM>
__device__ __forceinline__ bool gj_inverse(const float* v, float4* A, int M, int lane, const float* vlo = nullptr) {
  constexpr int MM = MAXM * MAXM;
  constexpr int R = MM > 32 ? MM / 32 : 1;
  constexpr int IG = 32 / MAXM;
  const int j = lane % MAXM, i0 = lane / MAXM;
  bool own[R];
  cdf a[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = i0 + r * IG;
    own[r] = lane < MM && i < M && j < M;
    float re = 0.f, im = 0.f, rl = 0.f, il = 0.f;
    if (own[r]) {
      const int ia = (i <= j) ? i * MAXM + j : j * MAXM + i;   // Re V_ij slot
      const int ib = (i <= j) ? j * MAXM + i : i * MAXM + j;   // Im slot (sign below)
      const float sg = (i <= j) ? 1.f : -1.f;
      re = v[ia];
      im = (i == j) ? 0.f : sg * v[ib];
      if (vlo) {
        rl = vlo[ia];
        il = (i == j) ? 0.f : sg * vlo[ib];
      }
    }
    a[r] = cdf{df{re, rl}, df{im, il}};
  }
  bool ok = true;
  for (int k = 0; k < M; ++k) {
    // A[i][k] of this lane's rows (lane i0 MAXM + k, slot r); A[k][j] and A[k][k] (lanes
    // (k % IG) MAXM + j and (k % IG) MAXM + k, slot k / IG)
    cdf col[R], row = cdf_zero(), piv = cdf_zero();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      col[r] = shfl_cdf(a[r], i0 * MAXM + k);
      const cdf rw = shfl_cdf(a[r], (k % IG) * MAXM + j);
      const cdf pv = shfl_cdf(a[r], (k % IG) * MAXM + k);
      if (k / IG == r) { row = rw; piv = pv; }
    }
    ok = ok && (piv.re.hi > 0.f) && isfinite(piv.re.hi);
    const df inv = df_rcp(piv.re);
    const cdf rs = cdf_scale(row, inv);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!own[r]) continue;
      const int i = i0 + r * IG;
      if (i == k && j == k) a[r] = cdf{inv, df{0.f, 0.f}};
      else if (i == k) a[r] = rs;
      else if (j == k) a[r] = cdf_scale(col[r], df_neg(inv));
      else a[r] = cdf_sub(a[r], cdf_mul(col[r], rs));
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (own[r]) A[(i0 + r * IG) * MAXM + j] = cdf_pack(a[r]);
  __syncwarp();
  return ok;
}

// The row sweep of the IP update for one bin (Eqs. 19-20), on one warp, with Q_f^-1 held
// in registers: lane l holds the entries (i, j) with j = l % MAXM and i = l / MAXM + r * IG
// (IG = 32 / MAXM, r < R; R = 2 for MAXM = 8, else 1, lanes >= MAXM^2 then idle).  Per row m:
//   c = Q_f^-1 e_m (shuffled from the lanes that hold column m),
//   q = T V_fm^-1 c              (sum over j: butterfly within the MAXM lanes of row i),
//   s = Re(c^H q),  u~ = q^H Q_f^-1   (both a sum over i: one butterfly across the rows),
//   r = 1/sqrt(s),  row m of Q_f <- (q r)^H,
//   Q_f^-1 <- Q_f^-1 - c (r u~ - e_m^T) r       (Sherman-Morrison),  log|det Q_f|^2 += log s.
// Entries outside M x M are zero and stay zero.  Q_f^-1 goes back to Qi_s at the end;
// returns the sum of log s in float-float (on every lane), sets bad when some s is not
// positive and finite.
template <int MAXM>
__device__ __forceinline__ df ip_rows(const float4 (*Vi)[MAXM * MAXM], float4* Q_s, float4* Qi_s, int M,
                                      df Tdf, int lane, int& bad) {
  constexpr int MM = MAXM * MAXM;
  constexpr int R = MM > 32 ? MM / 32 : 1;
  constexpr int IG = 32 / MAXM;
  constexpr int LIM = MM < 32 ? MM : 32;  // lanes taking part in the sums over i
  const int j = lane % MAXM, i0 = lane / MAXM;
  bool ok[R];
  cdf qi[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = i0 + r * IG;
    ok[r] = lane < MM && i < M && j < M;
    qi[r] = ok[r] ? cdf_unpack(Qi_s[i * MAXM + j]) : cdf_zero();
  }
  df s_row = df_make(1.f);  // lane m keeps s of row m (its log is taken after the sweep)
  for (int m = 0; m < M; ++m) {
    cdf v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = ok[r] ? cdf_unpack(Vi[m][(i0 + r * IG) * MAXM + j]) : cdf_zero();
    // c_j = Qi[j][m] (lane (j % IG) MAXM + m, slot j / IG), c_i = Qi[i][m] (lane i0 MAXM + m, slot r)
    cdf cj = cdf_zero(), ci[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const cdf a = shfl_cdf(qi[r], (j % IG) * MAXM + m);
      if (j / IG == r) cj = a;
      const cdf b = shfl_cdf(qi[r], i0 * MAXM + m);
      ci[r] = (lane < MM && i0 + r * IG < M) ? b : cdf_zero();
    }
    cdf q[R];
#pragma unroll
    for (int r = 0; r < R; ++r) q[r] = cdf_mul(v[r], cj);
#pragma unroll
    for (int o = 1; o < MAXM; o <<= 1)
#pragma unroll
      for (int r = 0; r < R; ++r) q[r] = cdf_add(q[r], shfl_xor_cdf(q[r], o));
    df a = df{0.f, 0.f};
    cdf b = cdf_zero();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      q[r] = cdf_scale(q[r], Tdf);
      a = df_add(a, cdf_cmul(ci[r], q[r]).re);
      b = cdf_add(b, cdf_cmul(q[r], qi[r]));
    }
    // a and b are the same on the MAXM lanes of a row: sum them over the rows
#pragma unroll
    for (int o = MAXM; o < LIM; o <<= 1) {
      a = df_add(a, shfl_xor_df(a, o));
      b = cdf_add(b, shfl_xor_cdf(b, o));
    }
    df sv = a;
    if (!(sv.hi > 0.f) || !isfinite(sv.hi)) { bad = 1; sv = df_make(1.f); }
    const df rs = df_rsqrt(sv);
    if (lane == m) s_row = sv;
    if (j == 0)
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (lane < MM && i0 + r * IG < M) Q_s[m * MAXM + i0 + r * IG] = cdf_pack(cdf_conj(cdf_scale(q[r], rs)));
    cdf uj = cdf_scale(b, rs);
    if (j == m) uj.re = df_sub(uj.re, df_make(1.f));
#pragma unroll
    for (int r = 0; r < R; ++r) qi[r] = cdf_sub(qi[r], cdf_scale(cdf_mul(ci[r], uj), rs));
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (ok[r]) Qi_s[(i0 + r * IG) * MAXM + j] = cdf_pack(qi[r]);
  // the M logs in parallel (lanes >= M hold log 1 = 0), added in row order on every lane
  const df lg = df_logf(s_row);
  df ld_add = df{0.f, 0.f};
  for (int m = 0; m < M; ++m) ld_add = df_add(ld_add, shfl_df(lg, m));
  return ld_add;
}

// With pf (dynamic shared memory for it given), the CTA prefetches at its start what the
// later phases read but the IP does not change: the bin's X and y~ rows (x~ part) and its
// g~ and W entries (normalisation), with cp.async, so those loads overlap the IP chain.
// With PR, the x~ part also forms P_n, R_n of its frames from the new x~, y~ and
// the normalised g~ (the factors of the next W update).  With ll_tail == 0 the bins'
// log-likelihood terms are left in llpart / logdet for a later kernel to add up.
// One warp per channel of the bucket (warps m < M run the Gauss-Jordan sweeps, warp 0 the
// row sweep; all of them the prefetch and the per-frame x~ / P / R / LL part), at most 64
// registers a thread: 2048 threads per SM, which keeps room for other contexts' kernels.
template <int MAXM>
__global__ void __launch_bounds__(32 * MAXM, 32 / MAXM) k_ip(Prob p, int S, int flags, int xt_mode, unsigned ctr, int pf,
                                                  float* __restrict__ PR, int ll_tail) {
  constexpr int MM = MAXM * MAXM;
  __shared__ float4 A_s[MAXM][MM];       // per warp m: sum_t x x^H / y~_m, then its inverse
  __shared__ float4 Q_s[MM], Qi_s[MM];
  __shared__ float vsum_s[MAXM][MM];      // packed split sums per m
  __shared__ double ld_s;
  __shared__ int bad_s;
  const int f = blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // warp index the compiler knows to be warp-uniform (branches on it need no reconvergence
  // handling around the shuffles of the single-warp stretches)
  const int warp_u = __shfl_sync(0xffffffffu, warp, 0);
  const int M = p.M, N = p.N, K = p.K, F = p.F;
  if (f >= F) return;
  // prefetch buffers: X row [T*M] complex, y~ row [T*M], g~ [N][M], W [N][K]
  extern __shared__ __align__(16) float ipsm[];
  const int TMq = p.T * M;
  float2* pf_x = reinterpret_cast<float2*>(ipsm);
  float* pf_y = ipsm + 2 * TMq;
  float* pf_g = pf_y + ((TMq + 3) & ~3);
  float* pf_w = pf_g + ((N * M + 3) & ~3);
  if (pf) {
    const size_t row = (size_t)f * TMq;
    if (xt_mode) {
      if ((TMq & 1) == 0)
        for (int e = tid; e < TMq / 2; e += blockDim.x)
          cpa16(reinterpret_cast<float*>(pf_x + 2 * e), reinterpret_cast<const float*>(p.X + row + 2 * e));
      else
        for (int e = tid; e < TMq; e += blockDim.x) cpa8(pf_x + e, p.X + row + e, true);
      if ((TMq & 3) == 0)
        for (int e = tid; e < TMq / 4; e += blockDim.x) cpa16(pf_y + 4 * e, p.yt + row + 4 * e);
      else
        for (int e = tid; e < TMq; e += blockDim.x) cpa4(pf_y + e, p.yt + row + e, true);
    }
    for (int e = tid; e < N * M; e += blockDim.x) cpa4(pf_g + e, p.G + ((size_t)(e / M) * F + f) * M + e % M, true);
    for (int e = tid; e < N * K; e += blockDim.x) cpa4(pf_w + e, p.W + (size_t)e * F + f, true);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  for (int e = tid; e < M * M; e += blockDim.x) {
    const int r = e / M, c = e % M;
    Q_s[r * MAXM + c] = p.Qx[(size_t)f * M * M + e];
    Qi_s[r * MAXM + c] = p.Qix[(size_t)f * M * M + e];
  }
  if (tid == 0) {
    ld_s = p.logdet[f];
    bad_s = 0;
  }
  if (flags & FLAG_DO_V) {
    // packed split sums (float32, fixed order over the splits)
    const size_t psz = (size_t)F * M * MM;
    for (int e = tid; e < M * MM; e += blockDim.x)
      vsum_s[e / MM][e % MM] = sum_splits(p.part + (size_t)f * M * MM + e, psz, S);
    __syncthreads();
    if (warp_u < M) {
      const bool ok = gj_inverse<MAXM>(vsum_s[warp_u], A_s[warp_u], M, lane);
      if (!ok && lane == 0) bad_s = 1;
    }
    __syncthreads();
    if (warp_u == 0) {
      int bad = 0;
      const df ld_add = ip_rows<MAXM>(A_s, Q_s, Qi_s, M, df_make((float)p.T), lane, bad);
      if (lane == 0) {
        ld_s += df_to_double(ld_add);
        if (bad) bad_s = 1;
      }
    }
    __syncthreads();
  }
  if (pf) asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();  // prefetched rows visible to every thread
  // phi normalisation and write-back
  __shared__ float phi_s;
  __shared__ float nu_s[64];
  __shared__ float2 qf_s[MM];  // the normalised Q_f in float32 (x~ of this bin's frames)
  if (warp_u == 0) {
    df ph = df_make(1.f), sq = df_make(1.f), isq = df_make(1.f);
    if (flags & FLAG_NORMALISE) {
      df tr = df{0.f, 0.f};
      for (int e = lane; e < M * M; e += 32) tr = df_add(tr, cdf_abs2(cdf_unpack(Q_s[(e / M) * MAXM + e % M])));
      for (int o = 16; o > 0; o >>= 1) tr = df_add(tr, shfl_xor_df(tr, o));
      ph = df_div(tr, df_make((float)M));
      sq = df_sqrt(ph);
      isq = df_rcp(sq);
    }
    for (int e = lane; e < M * M; e += 32) {
      const int r = e / M, c = e % M;
      const cdf q = cdf_scale(cdf_unpack(Q_s[r * MAXM + c]), isq);
      const cdf qi = cdf_scale(cdf_unpack(Qi_s[r * MAXM + c]), sq);
      p.Qx[(size_t)f * M * M + e] = cdf_pack(q);
      p.Qix[(size_t)f * M * M + e] = cdf_pack(qi);
      p.Qf[(size_t)f * M * M + e] = make_float2(q.re.hi, q.im.hi);
      qf_s[r * MAXM + c] = make_float2(q.re.hi, q.im.hi);
      p.Qinv[(size_t)f * M * M + e] = make_float2(qi.re.hi, qi.im.hi);
    }
    if (lane == 0) {
      phi_s = ph.hi;
      const double ld = ld_s - (double)M * df_to_double(df_logf(ph));
      p.logdet[f] = ld;
      p.phi[f] = ph.hi;
      if (bad_s) flag(p.status, ST_SINGULAR);
      if (!isfinite(ld)) flag(p.status, ST_NONFINITE);
    }
  }
  if (flags & FLAG_NORMALISE) {
    // g~_nf /= phi_f, then nu_nf = sum_m g~_nfm: g~_nf /= nu_nf, w_nkf *= nu_nf
    __syncthreads();
    const float fphi = phi_s;
    for (int n0 = 0; n0 < N; n0 += 64) {
      const int nn = min(64, N - n0);
      if (tid < nn) {
        float* gp = p.G + ((size_t)(n0 + tid) * F + f) * M;
        const float* gsrc = pf ? pf_g + (n0 + tid) * M : gp;
        float gv[MAXM];
        float nu = 0.f;
#pragma unroll
        for (int m = 0; m < MAXM; ++m)
          if (m < M) { gv[m] = gsrc[m] / fphi; nu += gv[m]; }
#pragma unroll
        for (int m = 0; m < MAXM; ++m)
          if (m < M) {
            gp[m] = gv[m] / nu;
            if (pf) pf_g[(n0 + tid) * M + m] = gv[m] / nu;  // the normalised g~ for P, R
          }
        nu_s[tid] = nu;
        if (!(nu > 0.f) || !isfinite(nu)) flag(p.status, ST_NONFINITE);
      }
      __syncthreads();
      for (int e = tid; e < nn * K; e += blockDim.x) {
        const int n = e / K, k = e - n * K;
        float* wp = p.W + ((size_t)(n0 + n) * K + k) * F + f;
        *wp = (pf ? pf_w[(n0 + n) * K + k] : *wp) * nu_s[n];
      }
      __syncthreads();
    }
  }
  if (!xt_mode) return;
  // x~ = |Q_f x_ft|^2 for this bin's frames with the new (normalised) Q_f, y~ /= phi_f,
  // and this bin's log-likelihood terms (Eq. 17); the last CTA adds the bins up
  __syncthreads();
  const int T = p.T;
  const float ph = phi_s;
  const bool exact = (M == MAXM);
  float part = 0.f;
  for (int t = tid; t < T; t += blockDim.x) {
    const size_t pt = (size_t)f * T + t;
    float2 x[MAXM];
    float yv[MAXM];
    if (pf) {
#pragma unroll
      for (int j = 0; j < MAXM; ++j) {
        x[j] = (j < M) ? pf_x[t * M + j] : make_float2(0.f, 0.f);
        yv[j] = (j < M) ? pf_y[t * M + j] : 1.f;
      }
    } else if (exact) {
#pragma unroll
      for (int q = 0; q < MAXM / 2; ++q) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p.X + pt * MAXM) + q);
        x[2 * q] = make_float2(v.x, v.y);
        x[2 * q + 1] = make_float2(v.z, v.w);
      }
#pragma unroll
      for (int m = 0; m < MAXM; ++m) yv[m] = p.yt[pt * MAXM + m];
    } else {
#pragma unroll
      for (int j = 0; j < MAXM; ++j) {
        x[j] = (j < M) ? __ldg(p.X + pt * M + j) : make_float2(0.f, 0.f);
        yv[j] = (j < M) ? p.yt[pt * M + j] : 1.f;
      }
    }
    float ls = 0.f;
    float xa[MAXM], ya[MAXM];
#pragma unroll
    for (int m = 0; m < MAXM; ++m) {
      xa[m] = 0.f;
      ya[m] = 0.f;
      if (m < M) {
        float re = 0.f, im = 0.f;
#pragma unroll
        for (int j = 0; j < MAXM; ++j) {
          if (j < M) {
            const float2 q = qf_s[m * MAXM + j];
            re = fmaf(q.x, x[j].x, fmaf(-q.y, x[j].y, re));
            im = fmaf(q.x, x[j].y, fmaf(q.y, x[j].x, im));
          }
        }
        const float xv = re * re + im * im;
        const float y = yv[m] / ph;
        p.yt[pt * M + m] = y;
        p.xt[pt * M + m] = xv;
        xa[m] = xv;
        ya[m] = y;
        ls += -xv / y - logf(y);
      }
    }
    part += ls;
    // the normalised g~ of this bin: its prefetch copy, or the values this CTA wrote (visible
    // after the barrier above)
    if (PR != nullptr)
      pr_point<MAXM>(xa, ya, M, N, pf ? pf_g : p.G + (size_t)f * M, pf ? (size_t)M : (size_t)F * M, PR,
                     (size_t)F * T, pt);
  }
  __shared__ double red_s[MAXM];
  for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
  if (lane == 0) red_s[warp] = (double)part;
  __syncthreads();
  if (tid == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red_s[w];
    p.llpart[f] = sum;
  }
  if (!ll_tail || !arrive_last(p.counters + ctr, (unsigned)F)) return;
  double sll = 0.0, sld = 0.0;
  for (int b = tid; b < F; b += blockDim.x) {
    sll += __ldcg(p.llpart + b);
    sld += __ldcg(p.logdet + b);
  }
  for (int off = 16; off > 0; off >>= 1) {
    sll += __shfl_xor_sync(0xffffffffu, sll, off);
    sld += __shfl_xor_sync(0xffffffffu, sld, off);
  }
  __shared__ double red2_s[2][MAXM];
  if (lane == 0) { red2_s[0][warp] = sll; red2_s[1][warp] = sld; }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, d = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += red2_s[0][w]; d += red2_s[1][w]; }
    const double ll = a + (double)T * d - (double)F * T * M * 1.1447298858494002;  // log(pi)
    *p.ll = ll;
    if (!isfinite(ll)) flag(p.status, ST_NONFINITE);
  }
}

// ---------------------------------------------------------------------------------
// x~ = |Q_f x_ft|^2 with the new (normalised) Q_f; y~ /= phi_f; log-likelihood (Eq. 17);
// extra CTAs (blockIdx.x >= n_pt_blocks) apply the mu normalisation, one warp per (n,k).
// ---------------------------------------------------------------------------------
constexpr int kPtsPerThread = 4;

template <int MAXM>
__global__ void __launch_bounds__(kThreads) k_xt_ll(Prob p, int n_pt_blocks, int apply_phi, int do_mu,
                                                    unsigned ctr, int ll_bins, float* __restrict__ PR) {
  const int tid = threadIdx.x;
  const int M = p.M, T = p.T, F = p.F;
  if ((int)blockIdx.x < n_pt_blocks) {
    const unsigned npts = (unsigned)F * (unsigned)T;  // < 2^31 (checked at init)
    const unsigned pt0 = blockIdx.x * (unsigned)(kThreads * kPtsPerThread);
    const unsigned pt_end = min(npts, pt0 + (unsigned)(kThreads * kPtsPerThread));
    // Q_f (and phi_f) of the block's bins in shared memory when they fit: the per-point
    // loads then go to the shared-memory pipe instead of the global load queue
    constexpr int kQs = 2048;
    __shared__ float2 qs[kQs];
    __shared__ float phs[kQs / 4];
    const int fa = (int)(pt0 / (unsigned)T), nfb = (int)((pt_end - 1) / (unsigned)T) - fa + 1;
    const bool q_smem = nfb * M * M <= kQs && nfb <= kQs / 4;
    if (q_smem) {
      for (int e = tid; e < nfb * M * M; e += kThreads) qs[e] = __ldg(p.Qf + (size_t)fa * M * M + e);
      for (int e = tid; e < nfb; e += kThreads) phs[e] = apply_phi ? __ldg(p.phi + fa + e) : 1.f;
    }
    __syncthreads();
    const bool exact = (M == MAXM);  // vector loads and stores of whole points
    float part = 0.f;
    for (int r = 0; r < kPtsPerThread; ++r) {
      const unsigned pt = pt0 + (unsigned)(r * kThreads + tid);
      if (pt >= pt_end) break;
      const int f = (int)(pt / (unsigned)T);
      const float2* xp = p.X + (size_t)pt * M;
      const float2* qp = q_smem ? qs + (f - fa) * M * M : p.Qf + (size_t)f * M * M;
      float2 x[MAXM];
      float yv[MAXM], xv[MAXM];
      if (exact) {
#pragma unroll
        for (int q = 0; q < MAXM / 2; ++q) {
          const float4 v = __ldg(reinterpret_cast<const float4*>(xp) + q);
          x[2 * q] = make_float2(v.x, v.y);
          x[2 * q + 1] = make_float2(v.z, v.w);
        }
        if (MAXM % 4 == 0) {
#pragma unroll
          for (int q = 0; q < MAXM / 4; ++q) {
            const float4 v = *reinterpret_cast<const float4*>(p.yt + (size_t)pt * MAXM + 4 * q);
            yv[4 * q] = v.x; yv[4 * q + 1] = v.y; yv[4 * q + 2] = v.z; yv[4 * q + 3] = v.w;
          }
        } else {
#pragma unroll
          for (int m = 0; m < MAXM; ++m) yv[m] = p.yt[(size_t)pt * MAXM + m];
        }
      } else {
#pragma unroll
        for (int j = 0; j < MAXM; ++j) {
          x[j] = (j < M) ? __ldg(xp + j) : make_float2(0.f, 0.f);
          yv[j] = (j < M) ? p.yt[(size_t)pt * M + j] : 1.f;
        }
      }
      const float ph = q_smem ? phs[f - fa] : (apply_phi ? p.phi[f] : 1.f);
      float ls = 0.f;
#pragma unroll
      for (int m = 0; m < MAXM; ++m) {
        xv[m] = 0.f;
        if (m < M) {
          float re = 0.f, im = 0.f;
#pragma unroll
          for (int j = 0; j < MAXM; ++j) {
            if (j < M) {
              const float2 q = qp[m * M + j];
              re = fmaf(q.x, x[j].x, fmaf(-q.y, x[j].y, re));
              im = fmaf(q.x, x[j].y, fmaf(q.y, x[j].x, im));
            }
          }
          xv[m] = re * re + im * im;
          if (apply_phi) yv[m] = yv[m] / ph;
          ls += -xv[m] / yv[m] - logf(yv[m]);
        }
      }
      if (exact && MAXM % 4 == 0) {
#pragma unroll
        for (int q = 0; q < MAXM / 4; ++q) {
          *reinterpret_cast<float4*>(p.xt + (size_t)pt * MAXM + 4 * q) =
              make_float4(xv[4 * q], xv[4 * q + 1], xv[4 * q + 2], xv[4 * q + 3]);
          if (apply_phi)
            *reinterpret_cast<float4*>(p.yt + (size_t)pt * MAXM + 4 * q) =
                make_float4(yv[4 * q], yv[4 * q + 1], yv[4 * q + 2], yv[4 * q + 3]);
        }
      } else {
#pragma unroll
        for (int m = 0; m < MAXM; ++m)
          if (m < M) {
            p.xt[(size_t)pt * M + m] = xv[m];
            if (apply_phi) p.yt[(size_t)pt * M + m] = yv[m];
          }
      }
      part += ls;
      // P, R of the next W update from this point's new x~, y~ and the bin's g~
      if (PR != nullptr) pr_point<MAXM>(xv, yv, M, p.N, p.G + (size_t)f * M, (size_t)F * M, PR, npts, pt);
    }
    // block reduction in a fixed order (float64 from the warp sums on)
    __shared__ double red[kThreads / 32];
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if ((tid & 31) == 0) red[tid >> 5] = (double)part;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) s += red[w];
      p.llpart[blockIdx.x] = s;
    }
    if (!arrive_last(p.counters + ctr, (unsigned)n_pt_blocks)) return;
    double s = 0.0;
    for (int b = tid; b < n_pt_blocks; b += kThreads) s += __ldcg(p.llpart + b);
    double ld = 0.0;
    for (int f = tid; f < F; f += kThreads) ld += __ldcg(p.logdet + f);
    __syncthreads();
    for (int off = 16; off > 0; off >>= 1) {
      s += __shfl_xor_sync(0xffffffffu, s, off);
      ld += __shfl_xor_sync(0xffffffffu, ld, off);
    }
    __shared__ double red2[2][kThreads / 32];
    if ((tid & 31) == 0) { red2[0][tid >> 5] = s; red2[1][tid >> 5] = ld; }
    __syncthreads();
    if (tid == 0) {
      double S = 0.0, LD = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) { S += red2[0][w]; LD += red2[1][w]; }
      const double ll = S + (double)T * LD - (double)F * T * M * 1.1447298858494002;  // log(pi)
      *p.ll = ll;
      if (!isfinite(ll)) flag(p.status, ST_NONFINITE);
    }
  } else if ((int)blockIdx.x < n_pt_blocks + (do_mu ? p.N * p.K : 0)) {
    // mu_nk = sum_f w_nkf;  w_nk /= mu;  h_nk *= mu   (one CTA per (n, k) row)
    const int nk = (int)blockIdx.x - n_pt_blocks;
    float* __restrict__ w = p.W + (size_t)nk * F;
    float* __restrict__ h = p.H + (size_t)nk * T;
    float part = 0.f;
    for (int f = tid; f < F; f += kThreads) part += w[f];
    __shared__ float red[kThreads / 32];
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if ((tid & 31) == 0) red[tid >> 5] = part;
    __syncthreads();
    float mu = 0.f;
    for (int i = 0; i < kThreads / 32; ++i) mu += red[i];
    const float inv = 1.f / mu;
    for (int f = tid; f < F; f += kThreads) w[f] *= inv;
    for (int t = tid; t < T; t += kThreads) h[t] *= mu;
    if (tid == 0 && !(mu > 0.f && isfinite(mu))) flag(p.status, ST_NONFINITE);
  } else if (ll_bins) {
    // the last block: the per-bin log-likelihood terms and log-dets that the IP kernel left,
    // added up in bin order (Eq. 17)
    double sll = 0.0, sld = 0.0;
    for (int b = tid; b < F; b += kThreads) {
      sll += __ldcg(p.llpart + b);
      sld += __ldcg(p.logdet + b);
    }
    for (int off = 16; off > 0; off >>= 1) {
      sll += __shfl_xor_sync(0xffffffffu, sll, off);
      sld += __shfl_xor_sync(0xffffffffu, sld, off);
    }
    __shared__ double red_ll[2][kThreads / 32];
    if ((tid & 31) == 0) { red_ll[0][tid >> 5] = sll; red_ll[1][tid >> 5] = sld; }
    __syncthreads();
    if (tid == 0) {
      double a = 0.0, d = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) { a += red_ll[0][w]; d += red_ll[1][w]; }
      const double ll = a + (double)T * d - (double)F * T * M * 1.1447298858494002;  // log(pi)
      *p.ll = ll;
      if (!isfinite(ll)) flag(p.status, ST_NONFINITE);
    }
  }
}

// ---------------------------------------------------------------------------------
// Per-bin preparation of a newly set state (init / set_state / restart), float64, one
// warp per bin: Q_f^-1 (Gauss-Jordan) and log|det Q_f|^2 (LU), stored in the float-float
// format the IP kernel carries across iterations; float32 copies; phi_f = 1.
// ---------------------------------------------------------------------------------
template <int MAXM>
__global__ void __launch_bounds__(kThreads) k_prep_q(Prob p) {
  __shared__ double2 A_s[kThreads / 32][MAXM * 2 * MAXM];
  __shared__ double2 fac_s[kThreads / 32][MAXM];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int f = blockIdx.x * (kThreads / 32) + warp;
  if (f >= p.F) return;
  const int M = p.M;
  double2* A = A_s[warp];
  const float4* q = p.Qx + (size_t)f * M * M;
  // log|det Q|^2
  for (int e = lane; e < M * M; e += 32) {
    const float4 v = q[e];
    A[(e / M) * MAXM + e % M] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
    p.Qf[(size_t)f * M * M + e] = make_float2(v.x, v.z);
  }
  __syncwarp();
  const double ld = warp_logdet2(M, MAXM, A, fac_s[warp]);
  // Q^-1
  const int LD = 2 * MAXM;
  for (int e = lane; e < M * 2 * M; e += 32) {
    const int r = e / (2 * M), c = e % (2 * M);
    if (c < M) {
      const float4 v = q[r * M + c];
      A[r * LD + c] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
    } else {
      A[r * LD + c] = make_double2(c - M == r ? 1.0 : 0.0, 0.0);
    }
  }
  __syncwarp();
  const bool ok = warp_gauss_jordan(M, M, LD, A, fac_s[warp]);
  for (int e = lane; e < M * M; e += 32) {
    const double2 v = A[(e / M) * LD + M + e % M];
    const df re = df_from_double(v.x), im = df_from_double(v.y);
    p.Qix[(size_t)f * M * M + e] = make_float4(re.hi, re.lo, im.hi, im.lo);
    p.Qinv[(size_t)f * M * M + e] = make_float2(re.hi, im.hi);
  }
  if (lane == 0) {
    p.logdet[f] = ld;
    p.phi[f] = 1.f;
    if (!ok || !isfinite(ld)) flag(p.status, ST_SINGULAR);
  }
}

// ---------------------------------------------------------------------------------
// Multichannel Wiener filter (Eq. 3 with Eq. 16 substituted):
//   x_ftn = Q_f^-1 ( lambda_ftn g~_nf / y~_ft  (elementwise)  Q_f x_ft )
// grid = (F tiles of kOT, T splits), lambda formed on chip as in k_tile.
// ---------------------------------------------------------------------------------
template <int MAXM>
__global__ void __launch_bounds__(kThreads) k_separate(Prob p, Geom g, float2* __restrict__ out) {
  extern __shared__ __align__(16) float sm[];
  const int tid = threadIdx.x;
  const int N = p.N, K = p.K, M = p.M, NK = N * K, F = p.F, T = p.T;
  const int o_base = blockIdx.x * kOT;
  const int n_own = min(kOT, F - o_base);
  const int i_begin = blockIdx.y * g.span;
  const int i_end = min(T, i_begin + g.span);
  const int IC = g.IC, ICP = g.ICP;
  // lambda materialised (mixed form): read per point instead of formed from W and H tiles
  const bool lam_mem = p.lam != nullptr;
  const int MM = MAXM * MAXM;
  float2* q_s = reinterpret_cast<float2*>(sm);   // [kOT][MAXM*MAXM] (rows padded to MAXM)
  float2* qi_s = q_s + kOT * MM;                  // [kOT][MAXM*MAXM]
  float* g_s = reinterpret_cast<float*>(qi_s + kOT * MM);   // [N][kOT][M]
  float* own_s = g_s + ((N * kOT * M + 3) & ~3);  // [NK][kOT]        (W, H tiles: not lam_mem)
  float* oth_s = own_s + NK * kOT;                 // [NK][ICP]
  float* lam_s = oth_s + NK * ICP;                 // [N][kOT][ICP]

  for (int e = tid; e < N * kOT * M; e += kThreads) {
    const int n = e / (kOT * M), o = (e / M) % kOT, m = e % M;
    g_s[e] = (o < n_own) ? p.G[((size_t)n * F + o_base + o) * M + m] : 0.f;
  }
  for (int e = tid; e < kOT * MM; e += kThreads) {
    const int o = e / MM, r = (e % MM) / MAXM, c = e % MAXM;
    const bool v = o < n_own && r < M && c < M;
    q_s[e] = v ? p.Qf[((size_t)(o_base + o) * M + r) * M + c] : make_float2(0.f, 0.f);
    qi_s[e] = v ? p.Qinv[((size_t)(o_base + o) * M + r) * M + c] : make_float2(0.f, 0.f);
  }
  if (!lam_mem)
    for (int e = tid; e < NK * kOT; e += kThreads) {
      const int nk = e / kOT, o = e % kOT;
      own_s[e] = (o < n_own) ? p.W[(size_t)nk * F + o_base + o] : 0.f;
    }
  for (int i0 = i_begin; i0 < i_end; i0 += IC) {
    const int icn = min(IC, i_end - i0);
    __syncthreads();
    if (!lam_mem) {
      for (int row = tid >> 5; row < NK; row += kThreads / 32) {
        const float* src = p.H + (size_t)row * T + i0;
        float* dst = oth_s + row * ICP;
        for (int i = tid & 31; i < IC; i += 32) dst[i] = (i < icn) ? src[i] : 0.f;
      }
      __syncthreads();
      const int nq = IC / 4;
      for (int it = tid; it < (kOT / 2) * nq; it += kThreads) {
        const int o0 = (it / nq) * 2, ii = (it % nq) * 4;
        for (int n = 0; n < N; ++n) {
          float lam[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
          for (int k = 0; k < K; ++k) {
            const int nk = n * K + k;
            const float2 w = *reinterpret_cast<const float2*>(own_s + nk * kOT + o0);
            const float4 h = ld4(oth_s + nk * ICP + ii);
            lam[0][0] = fmaf(w.x, h.x, lam[0][0]); lam[0][1] = fmaf(w.x, h.y, lam[0][1]);
            lam[0][2] = fmaf(w.x, h.z, lam[0][2]); lam[0][3] = fmaf(w.x, h.w, lam[0][3]);
            lam[1][0] = fmaf(w.y, h.x, lam[1][0]); lam[1][1] = fmaf(w.y, h.y, lam[1][1]);
            lam[1][2] = fmaf(w.y, h.z, lam[1][2]); lam[1][3] = fmaf(w.y, h.w, lam[1][3]);
          }
          st4(lam_s + (n * kOT + o0) * ICP + ii, make_float4(lam[0][0], lam[0][1], lam[0][2], lam[0][3]));
          st4(lam_s + (n * kOT + o0 + 1) * ICP + ii, make_float4(lam[1][0], lam[1][1], lam[1][2], lam[1][3]));
        }
      }
    }
    __syncthreads();
    // one point per thread (t fastest across lanes)
    for (int e = tid; e < kOT * IC; e += kThreads) {
      const int o = e / IC, i = e % IC;
      if (o >= n_own || i >= icn) continue;
      const int f = o_base + o, t = i0 + i;
      const size_t pt = (size_t)f * T + t;
      const bool exact = (M == MAXM);
      float2 x[MAXM], y[MAXM];
      if (exact) {
#pragma unroll
        for (int q = 0; q < MAXM / 2; ++q) {
          const float4 v = __ldg(reinterpret_cast<const float4*>(p.X + pt * MAXM) + q);
          x[2 * q] = make_float2(v.x, v.y);
          x[2 * q + 1] = make_float2(v.z, v.w);
        }
      } else {
#pragma unroll
        for (int j = 0; j < MAXM; ++j) x[j] = (j < M) ? __ldg(p.X + pt * M + j) : make_float2(0.f, 0.f);
      }
      // y = Q_f x (rows of Q read two entries at a time)
      const float4* Qo = reinterpret_cast<const float4*>(q_s + o * MM);
      const float4* Qi = reinterpret_cast<const float4*>(qi_s + o * MM);
#pragma unroll
      for (int m = 0; m < MAXM; ++m) {
        float sr = 0.f, si = 0.f;
#pragma unroll
        for (int j = 0; j < MAXM; j += 2) {
          const float4 q = Qo[(m * MAXM + j) >> 1];
          sr = fmaf(q.x, x[j].x, fmaf(-q.y, x[j].y, sr));
          si = fmaf(q.x, x[j].y, fmaf(q.y, x[j].x, si));
          sr = fmaf(q.z, x[j + 1].x, fmaf(-q.w, x[j + 1].y, sr));
          si = fmaf(q.z, x[j + 1].y, fmaf(q.w, x[j + 1].x, si));
        }
        y[m] = make_float2(sr, si);
      }
      auto lam_of = [&](int n) {
        return lam_mem ? __ldg(p.lam + ((size_t)n * F + f) * T + t) : lam_s[(n * kOT + o) * ICP + i];
      };
      float ytot[MAXM];
#pragma unroll
      for (int m = 0; m < MAXM; ++m) ytot[m] = 0.f;
      for (int n = 0; n < N; ++n) {
        const float l = lam_of(n);
#pragma unroll
        for (int m = 0; m < MAXM; ++m)
          if (m < M) ytot[m] = fmaf(l, g_s[(n * kOT + o) * M + m], ytot[m]);
      }
      float yinv[MAXM];
#pragma unroll
      for (int m = 0; m < MAXM; ++m) yinv[m] = (m < M) ? __fdividef(1.f, ytot[m]) : 0.f;
      for (int n = 0; n < N; ++n) {
        const float l = lam_of(n);
        float2 z[MAXM];
#pragma unroll
        for (int m = 0; m < MAXM; ++m) {
          const float gain = (m < M) ? l * g_s[(n * kOT + o) * M + m] * yinv[m] : 0.f;
          z[m] = make_float2(gain * y[m].x, gain * y[m].y);
        }
        float2 r[MAXM];
#pragma unroll
        for (int m = 0; m < MAXM; ++m) {
          float sr = 0.f, si = 0.f;
#pragma unroll
          for (int j = 0; j < MAXM; j += 2) {
            const float4 q = Qi[(m * MAXM + j) >> 1];
            sr = fmaf(q.x, z[j].x, fmaf(-q.y, z[j].y, sr));
            si = fmaf(q.x, z[j].y, fmaf(q.y, z[j].x, si));
            sr = fmaf(q.z, z[j + 1].x, fmaf(-q.w, z[j + 1].y, sr));
            si = fmaf(q.z, z[j + 1].y, fmaf(q.w, z[j + 1].x, si));
          }
          r[m] = make_float2(sr, si);
        }
        float2* op = out + (((size_t)n * F + f) * T + t) * M;
        if (exact) {
#pragma unroll
          for (int q = 0; q < MAXM / 2; ++q)
            reinterpret_cast<float4*>(op)[q] = make_float4(r[2 * q].x, r[2 * q].y, r[2 * q + 1].x, r[2 * q + 1].y);
        } else {
#pragma unroll
          for (int m = 0; m < MAXM; ++m)
            if (m < M) op[m] = r[m];
        }
      }
    }
  }
}

}  // namespace fm
