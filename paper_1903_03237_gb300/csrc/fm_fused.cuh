// Bin-fused FastMNMF / FastFCA iteration (plain FP32 arithmetic, float-float IP), included by
// fm_kernels_inst.cuh for each channel bucket MAXM.
//
// Of the blocks of one iteration (Sec. III, order W -> H -> g~ -> Q -> normalise), only the H
// update (Eq. 24) sums over frequency bins.  Everything else is independent per bin f:
//   g~ update (Eq. 21: sums over t), V_fm (Eq. 18: over t), the IP update of Q_f (Eqs. 19-20),
//   x~_ft = |Q_f x_ft|^2, the bin's terms of Eq. 17, the phi and nu normalisation, and the
//   W update of the next iteration (Eq. 23: w_nkf sums over t only).
// So an iteration is two launches:
//   k_hgemm the H update: sum_f w_nkf {P, R}_nft as a register-tiled FP32 GEMM per source,
//           split over bins, with the update applied by the last CTA of each tile;
//   k_bin   one CTA per bin: lambda_ftn = sum_k w_nkf h_nkt (Eq. 9) for the bin's frames, g~,
//           V_fm + IP, normalisation, x~, log-likelihood terms, the next W update, and the
//           per-point factors P, R of the next H update from the lambda of the new W (or,
//           for the unconstrained source model of FastFCA, the lambda update of Eq. 22
//           first, per point, and no W, H).
// The mu normalisation (w_nk /= mu_nk, h_nk *= mu_nk, mu_nk = sum_f w_nkf) leaves lambda, every
// ratio of the W and H rules and the log-likelihood unchanged, so it commutes with the
// updates: it is applied once at the end of a chunk of iterations (with the log-likelihood
// sum), which gives the state the per-iteration normalisation gives, up to rounding.
// Every sum has a fixed order (no atomics), so results are bitwise reproducible.
#pragma once
#include <cooperative_groups.h>

#include "fm_kernels.cuh"

namespace cg = cooperative_groups;

namespace fm {

// k_bin flags
enum : int {
  FU_G = 1,        // g~ update (Eq. 21)
  FU_Q = 2,        // V_fm and the IP update (Eqs. 18-20)
  FU_NORM = 4,     // phi and nu normalisation
  FU_W = 8,        // next W update (Eq. 23) from the new x~, g~, lambda
  FU_WONLY = 16,   // only the W update, from the state in memory (first of a chunk)
  FU_LAM = 32,     // unconstrained source model: lambda update (Eq. 22) before g~
  FU_LAMWB = 64,   // write lambda * nu back (lambda is the state, or no W update follows)
  FU_FREE = 128,   // unconstrained source model: lambda is the state (no W, H)
  FU_LAM0 = 256,   // form lambda of the bin from W, H first (NMF model)
  FU_PH = 512,     // end with P, R of the next H update (from the lambda of the new W)
  FU_PRSM = 1024,  // the W update's P, R in shared memory (2 N T floats after the layout)
  FU_LAMSM = 2048, // the bin's lambda in shared memory (N T floats after P, R) instead of lam
};

constexpr int kFuTC = 256;          // frames per chunk of k_bin (one per thread)
constexpr int kFuTCP = kFuTC + 1;   // padded chunk row: rows of different sources / channels
                                    // fall on different banks
constexpr int kFuMaxNM = 256;       // N*M limit of the fused schedule (the g~ sums: one thread per pair)

// Dynamic shared memory of k_bin, in floats.
struct BinSmem {
  int gs, ws, nu, lam, a, b, xr, xi, total;
};
__host__ __device__ inline BinSmem bin_smem(int N, int K, int maxm) {
  BinSmem s;
  int o = 0;
  s.gs = o; o += N * maxm;             // g~ of the bin [N][MAXM]
  s.ws = o; o += N * K;                // w of the bin [N][K]
  s.nu = o; o += N;                    // nu_nf
  o = (o + 3) & ~3;
  s.lam = o; o += N * kFuTCP;          // lambda of a chunk [N][TCP]
  s.a = o; o += maxm * kFuTCP;         // x~/y~^2 or 1/y~ of a chunk [MAXM][TCP]
  s.b = o; o += maxm * kFuTCP;         // 1/y~ [MAXM][TCP]
  s.xr = o; o += maxm * kFuTCP;        // Re x [MAXM][TCP]
  s.xi = o; o += maxm * kFuTCP;        // Im x [MAXM][TCP]
  s.total = o;                         // the reductions reuse a..xi (>= 4 MAXM TCP floats)
  return s;
}
// With FU_PRSM the W update's P, R [2N][T] follow the layout (16-byte aligned); with FU_LAMSM
// the bin's lambda [N][T] follows them (after the P, R space when FU_PRSM is set).
__host__ __device__ inline int bin_smem_pr_offset(int N, int K, int maxm) { return (bin_smem(N, K, maxm).total + 3) & ~3; }
__host__ __device__ inline int bin_smem_lam_offset(int N, int K, int maxm, int T, bool prsm) {
  return bin_smem_pr_offset(N, K, maxm) + (prsm ? ((2 * N * T + 3) & ~3) : 0);
}

// Correctly rounded reciprocal (the ratios of every MU rule).
__device__ __forceinline__ float fu_rcp(float y) { return __frcp_rn(y); }

// lambda_ftn = sum_k w_nkf h_nkt (Eq. 9) for the bin's frames, w of the bin in shared memory,
// into out[n * FT + t] (the bin's rows of lam, or of a shared-memory copy with FT = T).  Work
// items are (4-frame group, source) pairs (16-byte rows of H) when T is a multiple of 4, else
// (frame, source) pairs; the k sum in order.
__device__ __forceinline__ void bin_lambda(const Prob& p, const float* ws, float* out, size_t FT) {
  const int T = p.T, N = p.N, K = p.K, tid = threadIdx.x;
  if ((T & 3) == 0) {
    // one (4-frame group, source) pair a thread at a time: every thread has work
    const int ng = T >> 2;
    for (int e = tid; e < ng * N; e += kThreads) {
      const int n = e / ng, t4 = 4 * (e - n * ng);
      const float* hr = p.H + (size_t)n * K * T + t4;
      const float* w = ws + n * K;
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 8
      for (int k = 0; k < K; ++k) {
        const float4 h = __ldg(reinterpret_cast<const float4*>(hr + (size_t)k * T));
        const float wk = w[k];
        a.x = fmaf(wk, h.x, a.x);
        a.y = fmaf(wk, h.y, a.y);
        a.z = fmaf(wk, h.z, a.z);
        a.w = fmaf(wk, h.w, a.w);
      }
      *reinterpret_cast<float4*>(out + n * FT + t4) = a;
    }
  } else {
    for (int e = tid; e < T * N; e += kThreads) {
      const int n = e / T, t = e - n * T;
      const float* hr = p.H + (size_t)n * K * T + t;
      const float* w = ws + n * K;
      float a = 0.f;
#pragma unroll 8
      for (int k = 0; k < K; ++k) a = fmaf(w[k], __ldg(hr + (size_t)k * T), a);
      out[n * FT + t] = a;
    }
  }
}

// The W update's sums for one bin (Eq. 23) and the update itself: num/den[n][k] = sum_t h_nkt
// {P, R}_nt, w_nk <- w_nk sqrt(num/den) (into W and into ws).  Warp w owns k = w + 8 j,
// j < KW (KW a compile-time bound; invalid k are skipped per warp), for every source.  With T a
// multiple of 4 a lane takes 16-byte groups of frames, U groups (U * 128 frames) a step, so that
// U * KW row loads are in flight; otherwise single frames.
template <int KW>
__device__ __forceinline__ void w_sums(const Prob& p, const float* Pw, size_t pws, float* ws, int f) {
  constexpr int nwarps = kThreads / 32;
  constexpr int U = KW <= 2 ? 4 : KW <= 4 ? 2 : 1;
  const int T = p.T, N = p.N, K = p.K, F = p.F;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool vec = (T & 3) == 0;
  for (int kb = 0; kb < K; kb += nwarps * KW) {
    const int k0 = kb + warp;
    if (k0 >= K) continue;
    const int kv = min(KW, (K - k0 + nwarps - 1) / nwarps);  // valid k of this warp
    for (int n = 0; n < N; ++n) {
      const float* Pn = Pw + n * pws;
      const float* Rn = Pw + (N + n) * pws;
      const float* __restrict__ Hn = p.H + ((size_t)n * K + k0) * T;
      float an[KW], ad[KW];
#pragma unroll
      for (int j = 0; j < KW; ++j) { an[j] = 0.f; ad[j] = 0.f; }
      if (vec) {
        for (int t0 = 4 * lane; t0 < T; t0 += 128 * U) {
          float4 Pv[U], Rv[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int t4 = t0 + 128 * u;
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
            Pv[u] = t4 < T ? *reinterpret_cast<const float4*>(Pn + t4) : z4;
            Rv[u] = t4 < T ? *reinterpret_cast<const float4*>(Rn + t4) : z4;
          }
#pragma unroll
          for (int j = 0; j < KW; ++j) {
            if (j >= kv) break;
            const float* hj = Hn + (size_t)j * nwarps * T;
            float4 h[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int t4 = t0 + 128 * u;
              h[u] = t4 < T ? __ldg(reinterpret_cast<const float4*>(hj + t4)) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
              an[j] = fmaf(h[u].x, Pv[u].x, fmaf(h[u].y, Pv[u].y, fmaf(h[u].z, Pv[u].z, fmaf(h[u].w, Pv[u].w, an[j]))));
              ad[j] = fmaf(h[u].x, Rv[u].x, fmaf(h[u].y, Rv[u].y, fmaf(h[u].z, Rv[u].z, fmaf(h[u].w, Rv[u].w, ad[j]))));
            }
          }
        }
      } else {
        for (int t = lane; t < T; t += 32) {
          const float Pv = Pn[t], Rv = Rn[t];
#pragma unroll
          for (int j = 0; j < KW; ++j) {
            if (j >= kv) break;
            const float h = __ldg(Hn + (size_t)j * nwarps * T + t);
            an[j] = fmaf(h, Pv, an[j]);
            ad[j] = fmaf(h, Rv, ad[j]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < KW; ++j)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          an[j] += __shfl_xor_sync(0xffffffffu, an[j], o);
          ad[j] += __shfl_xor_sync(0xffffffffu, ad[j], o);
        }
      if (lane == 0)
#pragma unroll
        for (int j = 0; j < KW; ++j) {
          if (j >= kv) break;
          const int k = k0 + j * nwarps;
          const float w = ws[n * K + k] * sqrtf(an[j] / ad[j]);
          if (!isfinite(w)) flag(p.status, ST_NONFINITE);
          p.W[((size_t)n * K + k) * F + f] = w;
          ws[n * K + k] = w;  // this warp owns (n, k): the lambda of the new W reads it
        }
    }
  }
}

// ---------------------------------------------------------------------------------------
// k_bin: one CTA (256 threads) per bin f.  lam: [N][F][T] (the bin's lambda, formed here
// from W, H with FU_LAM0; for the unconstrained model, the state itself).  PR: [2N][F][T]
// scratch for P, R of the W update, then for those of the H update that follows.  Frames go
// in chunks of 256, one per thread, staged in shared memory where a contraction over them
// follows.
// ---------------------------------------------------------------------------------------
template <int MAXM>
__global__ void __launch_bounds__(kThreads, 4) k_bin(Prob p, float* __restrict__ lam, float* __restrict__ PR,
                                                    int flags) {
  constexpr int MM = MAXM * MAXM;
  extern __shared__ __align__(16) float bsm[];
  __shared__ float4 A_s[MAXM][MM];     // per warp m: V_fm sums, then their inverses
  __shared__ float4 Q_s[MM], Qi_s[MM];
  __shared__ float vsum_s[MAXM][MM];   // packed V_fm sums per m (high parts)
  __shared__ float vlo_s[MAXM][MM];    // and their low parts (float-float)
  __shared__ float2 qf_s[MM];          // normalised Q_f in float32 (x~)
  __shared__ double ld_s;
  __shared__ float phi_s;
  __shared__ int bad_s;
  __shared__ double llred_s[kThreads / 32];
  const int f = blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // the warp index as a value the compiler knows to be warp-uniform: branches on it are not
  // treated as divergent, so the shuffle-heavy single-warp stretches (Gauss-Jordan, IP row
  // sweep, phi normalisation) need no reconvergence handling.  In a build with clock64
  // stamps at the phase boundaries the row sweep took four to five times longer with the
  // plain index; in this kernel the launch time is the same either way (the other CTAs on
  // the SM fill the issue slots the single warp leaves).
  const int warp_u = __shfl_sync(0xffffffffu, warp, 0);
  const int F = p.F, T = p.T, M = p.M, N = p.N, K = p.K;
  if (f >= F) return;
  const BinSmem L = bin_smem(N, K, MAXM);
  float* gs = bsm + L.gs;
  float* ws = bsm + L.ws;
  float* nus = bsm + L.nu;
  float* lamc = bsm + L.lam;
  float* ac = bsm + L.a;
  float* bc = bsm + L.b;
  float* xr = bsm + L.xr;
  float* xi = bsm + L.xi;
  float* red = bsm + L.a;
  const size_t FT = (size_t)F * T;
  const size_t fT = (size_t)f * T;
  // the W update's P, R: rows of T in shared memory, or rows of the bin in PR (stride F T)
  const bool prsm = (flags & FU_PRSM) != 0;
  float* Pw = prsm ? bsm + bin_smem_pr_offset(N, K, MAXM) : PR + fT;
  const size_t pws = prsm ? (size_t)T : FT;
  // the bin's lambda: rows of T in shared memory, or rows of the bin in lam (stride F T)
  const bool lamsm = (flags & FU_LAMSM) != 0;
  float* lb = lamsm ? bsm + bin_smem_lam_offset(N, K, MAXM, T, prsm) : lam + fT;
  const size_t ls = lamsm ? (size_t)T : FT;
  const float2* __restrict__ Xf = p.X + fT * M;
  float* __restrict__ xtf = p.xt + fT * M;
  const bool free_model = (flags & FU_FREE) != 0;
  const bool wonly = (flags & FU_WONLY) != 0;

  for (int e = tid; e < N * MAXM; e += kThreads) {
    const int n = e / MAXM, m = e % MAXM;
    gs[e] = (m < M) ? p.G[((size_t)n * F + f) * M + m] : 0.f;
  }
  if (!free_model)
    for (int e = tid; e < N * K; e += kThreads) ws[e] = p.W[(size_t)e * F + f];
  for (int e = tid; e < N; e += kThreads) nus[e] = 1.f;
  if (flags & FU_Q)
    for (int e = tid; e < M * M; e += kThreads) {
      const int r = e / M, c = e % M;
      Q_s[r * MAXM + c] = p.Qx[(size_t)f * M * M + e];
      Qi_s[r * MAXM + c] = p.Qix[(size_t)f * M * M + e];
    }
  if (tid == 0) {
    ld_s = p.logdet[f];
    bad_s = 0;
    phi_s = 1.f;
  }
  __syncthreads();
  if (!free_model && (flags & FU_LAM0)) {
    bin_lambda(p, ws, lb, ls);
    __syncthreads();  // the bin's lambda (global) is read by this CTA's threads below
  }

  // ---- unconstrained source model: lambda_ftn *= sqrt(sum_m g~ x~/y~^2 / sum_m g~/y~) (Eq. 22)
  if (free_model && !wonly && (flags & FU_LAM)) {
    for (int t = tid; t < T; t += kThreads) {
      float y[MAXM], x[MAXM];
#pragma unroll
      for (int m = 0; m < MAXM; ++m) {
        y[m] = 0.f;
        x[m] = (m < M) ? xtf[(size_t)t * M + m] : 0.f;
      }
      for (int n = 0; n < N; ++n) {
        const float l = lb[n * ls + t];
#pragma unroll
        for (int m = 0; m < MAXM; ++m)
          if (m < M) y[m] = fmaf(l, gs[n * MAXM + m], y[m]);
      }
      float A[MAXM], B[MAXM];
#pragma unroll
      for (int m = 0; m < MAXM; ++m) {
        B[m] = (m < M) ? fu_rcp(y[m]) : 0.f;
        A[m] = x[m] * B[m] * B[m];
      }
      for (int n = 0; n < N; ++n) {
        float P = 0.f, R = 0.f;
#pragma unroll
        for (int m = 0; m < MAXM; ++m)
          if (m < M) {
            P = fmaf(gs[n * MAXM + m], A[m], P);
            R = fmaf(gs[n * MAXM + m], B[m], R);
          }
        float* lp = lb + n * ls + t;
        const float l = *lp * sqrtf(P / R);
        if (!isfinite(l)) flag(p.status, ST_NONFINITE);
        *lp = l;
      }
    }
    __syncthreads();  // the updated lambda (global) is read by this CTA's threads below
  }

  // ---- g~ update (Eq. 21): num/den[n][m] = sum_t lambda_ftn {x~/y~^2, 1/y~}_ftm
  if ((flags & FU_G) && !wonly) {
    const int NM = N * M;
    const int parts = NM >= kThreads ? 1 : kThreads / NM;
    const bool act = tid < parts * NM;
    const int pair = tid % NM, part = tid / NM;
    const int gn = pair / M, gm = pair % M;
    float num = 0.f, den = 0.f;
    for (int t0 = 0; t0 < T; t0 += kFuTC) {
      const int tc = min(kFuTC, T - t0);
      if (tid < tc) {
        const int t = t0 + tid;
        float y[MAXM];
#pragma unroll
        for (int m = 0; m < MAXM; ++m) y[m] = 0.f;
        for (int n = 0; n < N; ++n) {
          const float l = lb[n * ls + t];
          lamc[n * kFuTCP + tid] = l;
#pragma unroll
          for (int m = 0; m < MAXM; ++m)
            if (m < M) y[m] = fmaf(l, gs[n * MAXM + m], y[m]);
        }
#pragma unroll
        for (int m = 0; m < MAXM; ++m)
          if (m < M) {
            const float b = fu_rcp(y[m]);
            ac[m * kFuTCP + tid] = xtf[(size_t)t * M + m] * b * b;
            bc[m * kFuTCP + tid] = b;
          }
      }
      __syncthreads();
      if (act)
        for (int i = part; i < tc; i += parts) {
          const float l = lamc[gn * kFuTCP + i];
          num = fmaf(l, ac[gm * kFuTCP + i], num);
          den = fmaf(l, bc[gm * kFuTCP + i], den);
        }
      __syncthreads();
    }
    if (act) {
      red[2 * (part * NM + pair)] = num;
      red[2 * (part * NM + pair) + 1] = den;
    }
    __syncthreads();
    if (tid < NM) {
      float sn = 0.f, sd = 0.f;
      for (int q = 0; q < parts; ++q) {
        sn += red[2 * (q * NM + tid)];
        sd += red[2 * (q * NM + tid) + 1];
      }
      const int n = tid / M, m = tid % M;
      const float g = gs[n * MAXM + m] * sqrtf(sn / sd);
      if (!isfinite(g)) flag(p.status, ST_NONFINITE);
      gs[n * MAXM + m] = g;
    }
    __syncthreads();
  }

  // ---- V_fm = sum_t x_ft x_ft^H / y~_ftm (Eq. 18; the 1/T of Eq. 18 is applied in the row
  // sweep), with y~ from the new g~; then the IP update of Q_f (Eqs. 19-20).
  // Thread (entry e = (a, b) of the M x M matrix, part): entry (a, b) holds Re V_ab for a <= b
  // and Im V_ba for a > b (the packed layout of gj_inverse), summed for every channel m.
  // The sums reach the float-float Gauss-Jordan inverse unrounded (float-float across parts):
  // V_fm can be ill-conditioned (few frames per channel), and float32 storage of V alone
  // would cost its condition number times 2^-24.  In the 8-channel bucket, where a thread's
  // part covers a quarter of the frames, every term is also compensated (TwoSum); in the
  // smaller buckets a part covers 1/16 of the frames or less and sums plainly.
  if ((flags & FU_Q) && !wonly) {
    const int E = M * M;
    const int parts = kThreads / E;  // E <= 64
    const bool act = tid < parts * E;
    const int e = tid % E, part = tid / E;
    const int a = e / M, b = e % M;
    float acc[MAXM], cmp[MAXM];
#pragma unroll
    for (int m = 0; m < MAXM; ++m) { acc[m] = 0.f; cmp[m] = 0.f; }
    for (int t0 = 0; t0 < T; t0 += kFuTC) {
      const int tc = min(kFuTC, T - t0);
      if (tid < tc) {
        const int t = t0 + tid;
        float y[MAXM];
#pragma unroll
        for (int m = 0; m < MAXM; ++m) y[m] = 0.f;
        for (int n = 0; n < N; ++n) {
          const float l = lb[n * ls + t];
#pragma unroll
          for (int m = 0; m < MAXM; ++m)
            if (m < M) y[m] = fmaf(l, gs[n * MAXM + m], y[m]);
        }
#pragma unroll
        for (int m = 0; m < MAXM; ++m)
          if (m < M) {
            ac[m * kFuTCP + tid] = fu_rcp(y[m]);
            const float2 x = Xf[(size_t)t * M + m];
            xr[m * kFuTCP + tid] = x.x;
            xi[m * kFuTCP + tid] = x.y;
          }
      }
      __syncthreads();
      if (act)
        for (int i = part; i < tc; i += parts) {
          const float ar = xr[a * kFuTCP + i], ai = xi[a * kFuTCP + i];
          const float br = xr[b * kFuTCP + i], bi = xi[b * kFuTCP + i];
          // a <= b: Re(x_a conj x_b);  a > b: Im(x_b conj x_a)
          const float v = (a <= b) ? fmaf(ar, br, ai * bi) : fmaf(bi, ar, -(br * ai));
#pragma unroll
          for (int m = 0; m < MAXM; ++m)
            if (m < M) {
              if (MAXM == 8) {
                const df s = two_sum(acc[m], __fmul_rn(ac[m * kFuTCP + i], v));
                acc[m] = s.hi;
                cmp[m] += s.lo;
              } else {
                acc[m] = fmaf(ac[m * kFuTCP + i], v, acc[m]);
              }
            }
        }
      __syncthreads();
    }
    if (act)
#pragma unroll
      for (int m = 0; m < MAXM; ++m)
        if (m < M) {
          red[2 * ((part * M + m) * E + e)] = acc[m];
          red[2 * ((part * M + m) * E + e) + 1] = cmp[m];
        }
    __syncthreads();
    for (int o = tid; o < M * E; o += kThreads) {
      const int m = o / E, ee = o % E;
      df s = df{0.f, 0.f};
      for (int q = 0; q < parts; ++q) {
        const int r = 2 * ((q * M + m) * E + ee);
        s = df_add(s, fast_two_sum(red[r], red[r + 1]));
      }
      vsum_s[m][(ee / M) * MAXM + ee % M] = s.hi;
      vlo_s[m][(ee / M) * MAXM + ee % M] = s.lo;
    }
    __syncthreads();
    if (warp_u < M) {
      const bool ok = gj_inverse<MAXM>(vsum_s[warp_u], A_s[warp_u], M, lane, vlo_s[warp_u]);
      if (!ok && lane == 0) bad_s = 1;
    }
    __syncthreads();
    if (warp_u == 0) {
      int bad = 0;
      const df ld_add = ip_rows<MAXM>(A_s, Q_s, Qi_s, M, df_make((float)T), lane, bad);
      if (lane == 0) {
        ld_s += df_to_double(ld_add);
        if (bad) bad_s = 1;
      }
    }
    __syncthreads();
  }

  // ---- phi normalisation (Q_f /= sqrt(phi), Q_f^-1 *= sqrt(phi), g~ /= phi,
  // log|det Q_f|^2 -= M log phi) and the float32 Q_f the x~ part uses
  const bool qnew = !wonly && (flags & (FU_Q | FU_NORM));
  if (qnew) {
    if (!(flags & FU_Q))
      for (int e = tid; e < M * M; e += kThreads) {
        const int r = e / M, c = e % M;
        Q_s[r * MAXM + c] = p.Qx[(size_t)f * M * M + e];
        Qi_s[r * MAXM + c] = p.Qix[(size_t)f * M * M + e];
      }
    __syncthreads();
    if (warp_u == 0) {
      df ph = df_make(1.f), sq = df_make(1.f), isq = df_make(1.f);
      if (flags & FU_NORM) {
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
        p.Qinv[(size_t)f * M * M + e] = make_float2(qi.re.hi, qi.im.hi);
        qf_s[r * MAXM + c] = make_float2(q.re.hi, q.im.hi);
      }
      if (lane == 0) {
        phi_s = ph.hi;
        const double ld = ld_s - (double)M * df_to_double(df_logf(ph));
        ld_s = ld;
        p.logdet[f] = ld;
        p.phi[f] = ph.hi;
        if (bad_s) flag(p.status, ST_SINGULAR);
        if (!isfinite(ld)) flag(p.status, ST_NONFINITE);
      }
    }
    __syncthreads();
    if (flags & FU_NORM) {
      // g~_nf /= phi_f; nu_nf = sum_m g~_nfm; g~_nf /= nu_nf; w_nkf *= nu_nf (or lambda_ftn *= nu_nf)
      const float fphi = phi_s;
      for (int n = tid; n < N; n += kThreads) {
        float gv[MAXM];
        float nu = 0.f;
#pragma unroll
        for (int m = 0; m < MAXM; ++m)
          if (m < M) {
            gv[m] = gs[n * MAXM + m] / fphi;
            nu += gv[m];
          }
#pragma unroll
        for (int m = 0; m < MAXM; ++m)
          if (m < M) gs[n * MAXM + m] = gv[m] / nu;
        nus[n] = nu;
        if (p.nu_out) p.nu_out[(size_t)n * F + f] = nu;
        if (!(nu > 0.f) || !isfinite(nu)) flag(p.status, ST_NONFINITE);
      }
      __syncthreads();
      if (!free_model)
        for (int e = tid; e < N * K; e += kThreads) ws[e] *= nus[e / K];
    }
  }
  if (!wonly && (flags & (FU_G | FU_NORM)))
    for (int e = tid; e < N * M; e += kThreads) {
      const int n = e / M, m = e % M;
      p.G[((size_t)n * F + f) * M + m] = gs[n * MAXM + m];
    }
  __syncthreads();

  // ---- x~ = |Q_f x_ft|^2 with the new Q_f (read back when Q_f did not change), y~ from the
  // normalised g~ and lambda nu, the bin's terms of Eq. 17, and P_n, R_n of the W update.
  const bool doW = !free_model && (flags & FU_W);
  const bool lamwb = !wonly && (flags & FU_LAMWB) && (flags & FU_NORM);
  float llacc = 0.f;
  for (int t = tid; t < T; t += kThreads) {
    float xv[MAXM], y[MAXM];
    if (qnew) {
      float2 x[MAXM];
#pragma unroll
      for (int j = 0; j < MAXM; ++j) x[j] = (j < M) ? Xf[(size_t)t * M + j] : make_float2(0.f, 0.f);
#pragma unroll
      for (int m = 0; m < MAXM; ++m) {
        xv[m] = 0.f;
        if (m < M) {
          float re = 0.f, im = 0.f;
#pragma unroll
          for (int j = 0; j < MAXM; ++j)
            if (j < M) {
              const float2 q = qf_s[m * MAXM + j];
              re = fmaf(q.x, x[j].x, fmaf(-q.y, x[j].y, re));
              im = fmaf(q.x, x[j].y, fmaf(q.y, x[j].x, im));
            }
          xv[m] = re * re + im * im;
          xtf[(size_t)t * M + m] = xv[m];
        }
      }
    } else {
#pragma unroll
      for (int m = 0; m < MAXM; ++m) xv[m] = (m < M) ? xtf[(size_t)t * M + m] : 0.f;
    }
#pragma unroll
    for (int m = 0; m < MAXM; ++m) y[m] = 0.f;
    for (int n = 0; n < N; ++n) {
      float* lp = lb + n * ls + t;
      const float l = *lp * nus[n];
      if (lamwb) *lp = l;
#pragma unroll
      for (int m = 0; m < MAXM; ++m)
        if (m < M) y[m] = fmaf(l, gs[n * MAXM + m], y[m]);
    }
    if (!wonly)
#pragma unroll
      for (int m = 0; m < MAXM; ++m)
        if (m < M) llacc += -xv[m] / y[m] - logf(y[m]);
    if (doW) {
      float A[MAXM], B[MAXM];
#pragma unroll
      for (int m = 0; m < MAXM; ++m) {
        B[m] = (m < M) ? fu_rcp(y[m]) : 0.f;
        A[m] = xv[m] * B[m] * B[m];
      }
      for (int n = 0; n < N; ++n) {
        float P = 0.f, R = 0.f;
#pragma unroll
        for (int m = 0; m < MAXM; ++m)
          if (m < M) {
            P = fmaf(gs[n * MAXM + m], A[m], P);
            R = fmaf(gs[n * MAXM + m], B[m], R);
          }
        Pw[n * pws + t] = P;
        Pw[(N + n) * pws + t] = R;
      }
    }
  }
  if (!wonly) {
    // the bin's sum of -x~/y~ - log y~ (float per thread, float64 across warps in order)
    for (int o = 16; o > 0; o >>= 1) llacc += __shfl_xor_sync(0xffffffffu, llacc, o);
    if (lane == 0) llred_s[warp] = (double)llacc;
  }
  __syncthreads();  // also makes this CTA's P, R writes visible to all its threads
  if (!wonly && tid == 0) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += llred_s[w];
    p.llpart[f] = s;
    if (!qnew) p.logdet[f] = ld_s;
  }

  // ---- W update of the next iteration (Eq. 23): num/den[n][k] = sum_t h_nkt {P, R}_nft.
  // Warp w owns k = w, w + 8, ... of every source (KW = ceil(K/8) of them, a compile-time count
  // in w_sums); lanes stride the frames (coalesced H rows).  The lane sums are added by a
  // butterfly (fixed order).
  if (doW) {
    const int KW = (K + 7) / 8;
    switch (KW) {
      case 1: w_sums<1>(p, Pw, pws, ws, f); break;
      case 2: w_sums<2>(p, Pw, pws, ws, f); break;
      case 3: w_sums<3>(p, Pw, pws, ws, f); break;
      case 4: w_sums<4>(p, Pw, pws, ws, f); break;
      case 5: case 6: w_sums<6>(p, Pw, pws, ws, f); break;
      default: w_sums<8>(p, Pw, pws, ws, f); break;  // K <= 64 here; larger K loops inside
    }
  } else if (!free_model && !wonly && (flags & FU_NORM)) {
    for (int e = tid; e < N * K; e += kThreads) p.W[(size_t)e * F + f] = ws[e];
  }

  // ---- P, R of the H update that follows (Eq. 24), from the lambda of the new W (or, with
  // no W update, the lambda * nu written above), the normalised g~ and the new x~.  The W
  // update's P, R in PR are no longer needed: these replace them.
  if (!free_model && (flags & FU_PH)) {
    __syncthreads();  // the W sums have read PR; the new w is in ws
    if (doW) {
      bin_lambda(p, ws, lb, ls);
      __syncthreads();
    }
    for (int t = tid; t < T; t += kThreads) {
      float y[MAXM], A[MAXM], B[MAXM];
#pragma unroll
      for (int m = 0; m < MAXM; ++m) y[m] = 0.f;
      for (int n = 0; n < N; ++n) {
        const float l = lb[n * ls + t];
#pragma unroll
        for (int m = 0; m < MAXM; ++m)
          if (m < M) y[m] = fmaf(l, gs[n * MAXM + m], y[m]);
      }
#pragma unroll
      for (int m = 0; m < MAXM; ++m) {
        B[m] = (m < M) ? fu_rcp(y[m]) : 0.f;
        A[m] = (m < M) ? xtf[(size_t)t * M + m] * B[m] * B[m] : 0.f;
      }
      for (int n = 0; n < N; ++n) {
        float P = 0.f, R = 0.f;
#pragma unroll
        for (int m = 0; m < MAXM; ++m)
          if (m < M) {
            P = fmaf(gs[n * MAXM + m], A[m], P);
            R = fmaf(gs[n * MAXM + m], B[m], R);
          }
        PR[n * FT + fT + t] = P;
        PR[(N + n) * FT + fT + t] = R;
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// k_hgemm: the H update of Eq. 24 as a register-tiled FP32 GEMM per source n,
//   num[k][t] = sum_f w_nkf P_nft,   den[k][t] = sum_f w_nkf R_nft,
// with P, R (the H update's per-point factors, from the lambda of the new W) written by the
// bins' kernel.  A tile is 32 bases x 64 frames of one source; its bins are split over the
// S CTAs of one thread-block cluster (S set at launch: even, at most 8, the grid within about
// two CTAs per SM), each summing its bins in chunks of 32 with two chunks in flight
// (cp.async into alternating buffers, so the next chunk's loads overlap this chunk's FMAs;
// thread (ty, tx) owns bases 2ty, 2ty+1 and frames 4tx..4tx+3: per bin one 8-byte W load and
// two 16-byte P, R loads feed 16 FMAs).  The CTAs leave their partial tiles in shared memory;
// after a cluster barrier CTA r adds rows r, r + S, ... of all of them, in rank order,
// through distributed shared memory and applies h <- h sqrt(num/den); a second cluster
// barrier keeps every partial tile alive until it has been read.
// ---------------------------------------------------------------------------------------
constexpr int kHgKT = 32, kHgTT = 64, kHgFC = 32;  // tile bases, tile frames, bins per chunk
constexpr int kHgMaxS = 8;        // bin splits = CTAs per cluster (the portable cluster size)
constexpr int kHgWS = kHgKT + 2;  // W chunk row (even, for 8-byte loads)

template <int MAXM>  // one instance per channel-bucket translation unit (MAXM is not used)
__global__ void __launch_bounds__(kThreads) k_hgemm(Prob p, const float* __restrict__ PR, int span) {
  __shared__ __align__(16) float Ws[2][kHgFC][kHgWS];
  __shared__ __align__(16) float Ps[2][kHgFC][kHgTT];  // P chunks; buffer 0 then this CTA's num tile
  __shared__ __align__(16) float Rs[2][kHgFC][kHgTT];  // R chunks; buffer 0 then this CTA's den tile
  static_assert(kHgFC >= kHgKT, "buffer 0 must hold a 32-row partial tile");
  cg::cluster_group cluster = cg::this_cluster();
  const int S = (int)cluster.num_blocks();
  const int tid = threadIdx.x;
  const int F = p.F, T = p.T, N = p.N, K = p.K;
  const int n = blockIdx.z / S, s = (int)cluster.block_rank();
  const int k0 = blockIdx.y * kHgKT, t0 = blockIdx.x * kHgTT;
  const int fbeg = min(F, s * span), fend = min(F, fbeg + span);
  const size_t FT = (size_t)F * T;
  const int ty = tid >> 4, tx = tid & 15;
  const bool vecT = (T & 3) == 0;
  float num[2][4], den[2][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { num[a][b] = 0.f; den[a][b] = 0.f; }
  const float* __restrict__ Pn = PR + (size_t)n * FT;
  const float* __restrict__ Rn = PR + (size_t)(N + n) * FT;
  // the copies of one chunk into buffer b, as one cp.async group (zero fill outside the tile)
  auto load = [&](int f0, int fc, int b) {
    for (int e = tid; e < kHgFC * kHgKT; e += kThreads) {
      const int kk = e / kHgFC, ff = e % kHgFC;
      const bool ok = ff < fc && k0 + kk < K;
      cpa4(&Ws[b][ff][kk], p.W + (ok ? ((size_t)n * K + k0 + kk) * F + f0 + ff : 0), ok);
    }
    if (vecT) {
      for (int e = tid; e < kHgFC * kHgTT / 4; e += kThreads) {
        const int ff = e / (kHgTT / 4), q = (e % (kHgTT / 4)) * 4;
        if (ff < fc && t0 + q < T) {
          const size_t o = (size_t)(f0 + ff) * T + t0 + q;
          cpa16(&Ps[b][ff][q], Pn + o);
          cpa16(&Rs[b][ff][q], Rn + o);
        } else {
          *reinterpret_cast<float4*>(&Ps[b][ff][q]) = make_float4(0.f, 0.f, 0.f, 0.f);
          *reinterpret_cast<float4*>(&Rs[b][ff][q]) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
    } else {
      for (int e = tid; e < kHgFC * kHgTT; e += kThreads) {
        const int ff = e / kHgTT, q = e % kHgTT;
        const bool ok = ff < fc && t0 + q < T;
        const size_t o = ok ? (size_t)(f0 + ff) * T + t0 + q : 0;
        cpa4(&Ps[b][ff][q], Pn + o, ok);
        cpa4(&Rs[b][ff][q], Rn + o, ok);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  const int nch = (fend - fbeg + kHgFC - 1) / kHgFC;
  if (nch > 0) load(fbeg, min(kHgFC, fend - fbeg), 0);
  for (int c = 0; c < nch; ++c) {
    const int b = c & 1;
    const int f0 = fbeg + c * kHgFC, fc = min(kHgFC, fend - f0);
    if (c + 1 < nch) {
      load(f0 + kHgFC, min(kHgFC, fend - f0 - kHgFC), b ^ 1);  // buffer b^1 was released below
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();  // chunk c visible to every thread
#pragma unroll 4
    for (int ff = 0; ff < fc; ++ff) {
      const float2 w = *reinterpret_cast<const float2*>(&Ws[b][ff][2 * ty]);
      const float4 pv = *reinterpret_cast<const float4*>(&Ps[b][ff][4 * tx]);
      const float4 rv = *reinterpret_cast<const float4*>(&Rs[b][ff][4 * tx]);
      const float pa[4] = {pv.x, pv.y, pv.z, pv.w}, ra[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        num[0][q] = fmaf(w.x, pa[q], num[0][q]);
        num[1][q] = fmaf(w.y, pa[q], num[1][q]);
        den[0][q] = fmaf(w.x, ra[q], den[0][q]);
        den[1][q] = fmaf(w.y, ra[q], den[1][q]);
      }
    }
    __syncthreads();  // buffer b is read: the load two chunks on may overwrite it
  }
  // this CTA's partial tiles into buffer 0 (row = base within the tile)
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    *reinterpret_cast<float4*>(&Ps[0][2 * ty + a][4 * tx]) = make_float4(num[a][0], num[a][1], num[a][2], num[a][3]);
    *reinterpret_cast<float4*>(&Rs[0][2 * ty + a][4 * tx]) = make_float4(den[a][0], den[a][1], den[a][2], den[a][3]);
  }
  cluster.sync();
  {
    // rows s, s + S, ... of the tile: one (base, frame) per thread and pass, the splits added
    // in rank order
    const int tt = tid % kHgTT;
    for (int kk = s + (tid / kHgTT) * S; kk < kHgKT; kk += (kThreads / kHgTT) * S) {
      float sn = 0.f, sd = 0.f;
#pragma unroll
      for (int q = 0; q < kHgMaxS; ++q) {
        if (q < S) {
          const float* rp = cluster.map_shared_rank(&Ps[0][0][0], q);
          const float* rr = cluster.map_shared_rank(&Rs[0][0][0], q);
          sn += rp[kk * kHgTT + tt];
          sd += rr[kk * kHgTT + tt];
        }
      }
      const int k = k0 + kk, t = t0 + tt;
      if (k < K && t < T) {
        const size_t i = ((size_t)n * K + k) * T + t;
        const float h = p.H[i] * sqrtf(sn / sd);
        if (!isfinite(h)) flag(p.status, ST_NONFINITE);
        p.H[i] = h;
      }
    }
  }
  cluster.sync();  // the other CTAs may still be reading this CTA's tiles
}

}  // namespace fm
