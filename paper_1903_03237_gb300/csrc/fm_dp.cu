// FastMNMF-DP kernels (Sec. III-B-3 and Sec. III-C-3 of arXiv 1903.03237): the deep-prior
// speech source lambda_ft0 = u_f v_t [sigma^2_theta(z_t)]_f with the decoder
// sigma^2_theta(z) = exp(W2 tanh(W1 z + b1) + b2), and NMF noise sources (Eq. 9) for
// n = 1..N-1.  The spatial part (g~ of Eq. 21, V_fm and the IP of Eqs. 18-20, the phi / nu
// normalisation, x~ and the terms of Eq. 17) is k_bin of the unconstrained source model on the
// same lambda; these kernels update the source-model parameters in between:
//
//   k_dp_mh      Metropolis sampling of z_t: S proposals per frame, all with y~^{-0}, g~ and
//                x~ of the iteration's start, so the frames are independent and one CTA runs
//                all S proposals of its frames with their inputs staged in shared memory
//   k_dp_fsweep  per bin f: the u_f rule, or the noise W rule (Eq. 23), then lambda of the bin
//   k_dp_tsweep  per tile of frames: the v_t rule, or the noise H rule (Eq. 24), then lambda
//   k_dp_norm    nu (from k_bin) into u and the noise W, then mu_0 = sum_f u_f and
//                mu_nk = sum_f w_nkf into v and H (lambda unchanged)
//   k_dp_init    r = sigma^2(z) and lambda of every source from the state
//
// All FP32 on the CUDA cores; sums in a fixed order (no atomics on values), so results are
// reproducible bit for bit.
#include <cuda_runtime.h>

#include "fm_launch.h"

namespace fm {
namespace {

constexpr int kDpTT = 2;                  // frames per CTA of the per-frame sweeps
constexpr int kDpFC = kThreads / kDpTT;   // bins per chunk of the per-frame sweeps (128)
constexpr int kDpMaxPairs = 256;          // (N-1) K noise bases per sweep CTA
constexpr int kDpItems = kDpMaxPairs * kDpTT / kThreads;  // H-sweep items per thread (2)
constexpr int kMhMaxThreads = 576;       // Metropolis CTA: one bin per thread up to F = 576


// Shared-memory layout (floats) of the Metropolis kernel for TB frames.
struct MhLayout {
  int xs, yr, g0, uf, rold, rnew, h, zs, zn, vs, red, total;
};
__host__ __device__ inline MhLayout mh_layout(int F, int M, int TB, int D, int Hd) {
  MhLayout L;
  int o = 0;
  auto take = [&](int n) { const int at = o; o += (n + 3) & ~3; return at; };
  L.xs = take(TB * M * F);     // x~ [tb*M + m][f]
  L.yr = take(TB * M * F);     // y~^{-0} [tb*M + m][f]
  L.g0 = take(M * F);          // g~_0 [m][f]
  L.uf = take(F);              // u_f
  L.rold = take(TB * F);       // r of the current z [tb][f]
  L.rnew = take(TB * F);       // r of the proposal
  L.h = take(TB * Hd);         // hidden layer [tb][j] (16-byte rows: Hd % 4 == 0)
  L.zs = take(TB * D);         // z [tb][d]
  L.zn = take(TB * D);         // proposal
  L.vs = take(TB);             // v_t
  L.red = take((kMhMaxThreads / 32) * TB);
  L.total = o;
  return L;
}

// y~ of one TF bin: y_m = sum_n lambda_nft g~_nfm (g~ of the bin in shared memory [n][MAXM]).
template <int MAXM>
__device__ __forceinline__ void bin_y(const float* __restrict__ lam, const float* gs, int N, int M, size_t FT,
                                      size_t ft, float (&y)[MAXM]) {
#pragma unroll
  for (int m = 0; m < MAXM; ++m) y[m] = 0.f;
  for (int n = 0; n < N; ++n) {
    const float l = lam[n * FT + ft];
#pragma unroll
    for (int m = 0; m < MAXM; ++m)
      if (m < M) y[m] = fmaf(l, gs[n * MAXM + m], y[m]);
  }
}

// The hidden layer of nt frames: h[tb][j] = tanh(b1_j + sum_d W1[j][d] z[tb][d]).
__device__ __forceinline__ void hidden_layer(const float* __restrict__ W1, const float* __restrict__ b1,
                                             const float* z, float* h, int nt, int D, int Hd) {
  for (int e = threadIdx.x; e < nt * Hd; e += blockDim.x) {
    const int tb = e / Hd, j = e - tb * Hd;
    float a = b1[j];
    const float* w = W1 + (size_t)j * D;
    for (int d = 0; d < D; ++d) a = fmaf(w[d], z[tb * D + d], a);
    h[tb * Hd + j] = tanhf(a);
  }
}

// The decoder's output layer for bin f and TB frames: s[tb] = b2_f + W2_f . h[tb].
template <int TB>
__device__ __forceinline__ void decode_bin(const float* __restrict__ W2, const float* __restrict__ b2,
                                           const float* h, int Hd, int f, float (&s)[TB]) {
  const float4* w = reinterpret_cast<const float4*>(W2 + (size_t)f * Hd);
#pragma unroll
  for (int i = 0; i < TB; ++i) s[i] = 0.f;
#pragma unroll 4
  for (int j4 = 0; j4 < (Hd >> 2); ++j4) {
    const float4 wv = __ldg(w + j4);
#pragma unroll
    for (int i = 0; i < TB; ++i) {
      const float4 hv = *reinterpret_cast<const float4*>(h + i * Hd + 4 * j4);
      s[i] = fmaf(wv.x, hv.x, s[i]);
      s[i] = fmaf(wv.y, hv.y, s[i]);
      s[i] = fmaf(wv.z, hv.z, s[i]);
      s[i] = fmaf(wv.w, hv.w, s[i]);
    }
  }
  const float b = b2[f];
#pragma unroll
  for (int i = 0; i < TB; ++i) s[i] += b;
}

// ---------------------------------------------------------------------------------------
// k_dp_init: r_t = sigma^2(z_t) into R[f][t] and lambda_ft0 = u_f v_t r_tf for TB frames per
// CTA; the noise sources' lambda_ftn = sum_k w_nkf h_nkt by k_dp_lam_noise.
// ---------------------------------------------------------------------------------------
template <int TB>
__global__ void __launch_bounds__(kThreads) k_dp_init(DpArgs a) {
  extern __shared__ __align__(16) float dsm[];
  const int F = a.p.F, T = a.p.T, D = a.D, Hd = a.Hd;
  const int t0 = blockIdx.x * TB, nt = min(TB, T - t0);
  float* h = dsm;                  // [TB][Hd]
  float* z = dsm + TB * Hd;        // [TB][D]
  for (int e = threadIdx.x; e < TB * Hd; e += kThreads) h[e] = 0.f;
  for (int e = threadIdx.x; e < nt * D; e += kThreads) z[e] = a.Z[(size_t)t0 * D + e];
  __syncthreads();
  hidden_layer(a.W1, a.b1, z, h, nt, D, Hd);
  __syncthreads();
  for (int f = threadIdx.x; f < F; f += kThreads) {
    float s[TB];
    decode_bin<TB>(a.W2, a.b2, h, Hd, f, s);
    const float uf = a.u[f];
#pragma unroll
    for (int tb = 0; tb < TB; ++tb)
      if (tb < nt) {
        const float r = expf(s[tb]);
        const size_t i = (size_t)f * T + t0 + tb;
        a.R[i] = r;
        a.lam[i] = uf * a.v[t0 + tb] * r;
        if (!isfinite(r)) flag(a.p.status, ST_NONFINITE);
      }
  }
}

__global__ void __launch_bounds__(kThreads) k_dp_lam_noise(DpArgs a) {
  const int F = a.p.F, T = a.p.T, N = a.p.N, K = a.K;
  const size_t FT = (size_t)F * T;
  const size_t i = (size_t)blockIdx.x * kThreads + threadIdx.x;
  if (i >= FT) return;
  const int f = (int)(i / T), t = (int)(i - (size_t)f * T);
  for (int n = 1; n < N; ++n) {
    float l = 0.f;
    for (int k = 0; k < K; ++k)
      l = fmaf(a.Wn[((size_t)(n - 1) * K + k) * F + f], a.Hn[((size_t)(n - 1) * K + k) * T + t], l);
    a.lam[n * FT + i] = l;
  }
}

// ---------------------------------------------------------------------------------------
// k_dp_mh: S Metropolis proposals for each of the CTA's TB frames (Sec. III-B-3).  With
// y~^{-0}_ftm = sum_{n>=1} lambda_ftn g~_nfm fixed, the log acceptance ratio of frame t is
//   log gamma_t = sum_{f,m} [ x~ (y_new - y_old) / (y_new y_old) - log(y_new / y_old) ],
//   y_old = lambda_old g~_0 + y~^{-0},  y_new = y_old + (lambda_new - lambda_old) g~_0,
// the change of Eq. 17 when lambda_ft0 alone changes (each term formed from the difference,
// so nothing cancels between two large sums).  Accepted where log u < log gamma_t.
// ---------------------------------------------------------------------------------------
template <int MAXM, int TB>
__global__ void __launch_bounds__(kMhMaxThreads) k_dp_mh(DpArgs a) {
  extern __shared__ __align__(16) float dsm[];
  __shared__ int acc_s[TB];
  const int F = a.p.F, T = a.p.T, M = a.p.M, N = a.p.N, D = a.D, Hd = a.Hd;
  const size_t FT = (size_t)F * T;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nthr = blockDim.x;
  const int t0 = blockIdx.x * TB, nt = min(TB, T - t0);
  const MhLayout L = mh_layout(F, M, TB, D, Hd);
  float* xs = dsm + L.xs;
  float* yr = dsm + L.yr;
  float* g0 = dsm + L.g0;
  float* uf = dsm + L.uf;
  float* rold = dsm + L.rold;
  float* rnew = dsm + L.rnew;
  float* h = dsm + L.h;
  float* zs = dsm + L.zs;
  float* zn = dsm + L.zn;
  float* vs = dsm + L.vs;
  float* red = dsm + L.red;

  // ---- stage the frames' x~, y~^{-0}, r and z, and the bins' g~_0 and u
  const int run = nt * M;  // x~ of the tile's frames is contiguous per bin
  for (int e = tid; e < F * run; e += nthr) {
    const int f = e / run, r = e - f * run, tb = r / M, m = r - tb * M;
    const size_t ft = (size_t)f * T + t0 + tb;
    xs[(tb * M + m) * F + f] = a.p.xt[ft * M + m];
    float y = 0.f;
    for (int n = 1; n < N; ++n) y = fmaf(a.lam[n * FT + ft], a.p.G[((size_t)n * F + f) * M + m], y);
    yr[(tb * M + m) * F + f] = y;
  }
  for (int e = tid; e < F * M; e += nthr) {
    const int f = e / M, m = e - f * M;
    g0[m * F + f] = a.p.G[(size_t)f * M + m];
  }
  for (int f = tid; f < F; f += nthr) {
    uf[f] = a.u[f];
    for (int tb = 0; tb < nt; ++tb) rold[tb * F + f] = a.R[(size_t)f * T + t0 + tb];
  }
  for (int e = tid; e < TB * Hd; e += nthr) h[e] = 0.f;  // rows of absent frames stay 0
  for (int e = tid; e < nt * D; e += nthr) zs[e] = a.Z[(size_t)t0 * D + e];
  if (tid < nt) vs[tid] = a.v[t0 + tid];
  unsigned n_acc = 0;
  __syncthreads();

  for (int s = 0; s < a.S; ++s) {
    // proposal z' = z + sqrt(eps) xi
    const float* xi = a.xi + ((size_t)s * T + t0) * D;
    for (int e = tid; e < nt * D; e += nthr) zn[e] = fmaf(a.sqrt_eps, xi[e], zs[e]);
    __syncthreads();
    hidden_layer(a.W1, a.b1, zn, h, nt, D, Hd);
    __syncthreads();
    float part[TB];
#pragma unroll
    for (int tb = 0; tb < TB; ++tb) part[tb] = 0.f;
    for (int f = tid; f < F; f += nthr) {
      float sv[TB];
      decode_bin<TB>(a.W2, a.b2, h, Hd, f, sv);
      const float u = uf[f];
#pragma unroll
      for (int tb = 0; tb < TB; ++tb)
        if (tb < nt) {
          const float rn = expf(sv[tb]);
          rnew[tb * F + f] = rn;
          const float lo = u * vs[tb] * rold[tb * F + f];
          const float dl = u * vs[tb] * rn - lo;
          float acc = 0.f;
#pragma unroll
          for (int m = 0; m < MAXM; ++m)
            if (m < M) {
              const float g = g0[m * F + f];
              const float yo = fmaf(lo, g, yr[(tb * M + m) * F + f]);
              const float d = dl * g;
              const float yn = yo + d;
              acc += xs[(tb * M + m) * F + f] * d / (yn * yo) - log1pf(d / yo);
            }
          part[tb] += acc;
        }
    }
    // log gamma per frame: warp sums, then the warps in order
#pragma unroll
    for (int tb = 0; tb < TB; ++tb) {
      float v = part[tb];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp * TB + tb] = v;
    }
    __syncthreads();
    if (tid < nt) {
      float lg = 0.f;
      for (int w = 0; w < (nthr >> 5); ++w) lg += red[w * TB + tid];
      const int acc = a.logu[(size_t)s * T + t0 + tid] < lg;
      acc_s[tid] = acc;
      n_acc += acc;
      if (a.loggamma) a.loggamma[(size_t)s * T + t0 + tid] = lg;
      if (isnan(lg)) flag(a.p.status, ST_NONFINITE);
    }
    __syncthreads();
    // accepted frames take the proposal (each thread copies what it wrote or will read)
    for (int e = tid; e < nt * D; e += nthr)
      if (acc_s[e / D]) zs[e] = zn[e];
    for (int f = tid; f < F; f += nthr)
#pragma unroll
      for (int tb = 0; tb < TB; ++tb)
        if (tb < nt && acc_s[tb]) rold[tb * F + f] = rnew[tb * F + f];
    __syncthreads();
  }

  // ---- the sampled z, its r and lambda_ft0 of the tile's frames
  for (int e = tid; e < nt * D; e += nthr) a.Z[(size_t)t0 * D + e] = zs[e];
  for (int f = tid; f < F; f += nthr)
    for (int tb = 0; tb < nt; ++tb) {
      const size_t i = (size_t)f * T + t0 + tb;
      const float r = rold[tb * F + f];
      a.R[i] = r;
      a.lam[i] = uf[f] * vs[tb] * r;
    }
  if (tid < nt && n_acc) atomicAdd(a.n_acc, (unsigned long long)n_acc);
}

// Block sum of two values in a fixed order (warp shuffles, then the warps in order); the
// result is returned to every thread.
__device__ __forceinline__ float2 block_sum2(float a, float b, float* red) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[2 * warp] = a;
    red[2 * warp + 1] = b;
  }
  __syncthreads();
  float2 s = make_float2(0.f, 0.f);
  for (int w = 0; w < kThreads / 32; ++w) {
    s.x += red[2 * w];
    s.y += red[2 * w + 1];
  }
  __syncthreads();
  return s;
}

// ---------------------------------------------------------------------------------------
// k_dp_fsweep: one CTA per bin f.  A_ftm = x~/y~^2, B_ftm = 1/y~ from the current lambda.
//  mode 0: u_f <- u_f sqrt( sum_t v_t r_tf P0_ft / sum_t v_t r_tf R0_ft ),
//          P0 = sum_m g~_0fm A, R0 = sum_m g~_0fm B; then lambda_ft0 = u_f v_t r_tf;
//  mode 1: w_nkf <- w_nkf sqrt( sum_t h_nkt Pn_ft / sum_t h_nkt Rn_ft ) for n >= 1 (Eq. 23);
//          then lambda_ftn = sum_k w_nkf h_nkt.
// ---------------------------------------------------------------------------------------
template <int MAXM>
__global__ void __launch_bounds__(kThreads) k_dp_fsweep(DpArgs a, int mode) {
  __shared__ float gs[8 * MAXM];      // g~ of the bin [n][MAXM] (N <= 8)
  __shared__ float red[2 * (kThreads / 32)];
  __shared__ float ws[kDpMaxPairs];
  __shared__ float Ps[7][kThreads], Rs[7][kThreads];
  __shared__ float uf_s;
  const int F = a.p.F, T = a.p.T, M = a.p.M, N = a.p.N, K = a.K;
  const size_t FT = (size_t)F * T;
  const int f = blockIdx.x, tid = threadIdx.x;
  for (int e = tid; e < N * MAXM; e += kThreads) {
    const int n = e / MAXM, m = e - n * MAXM;
    gs[e] = (m < M) ? a.p.G[((size_t)n * F + f) * M + m] : 0.f;
  }
  __syncthreads();
  const float* xtf = a.p.xt + (size_t)f * T * M;
  if (mode == 0) {
    float num = 0.f, den = 0.f;
    for (int t = tid; t < T; t += kThreads) {
      float y[MAXM];
      bin_y<MAXM>(a.lam, gs, N, M, FT, (size_t)f * T + t, y);
      float P = 0.f, Rr = 0.f;
#pragma unroll
      for (int m = 0; m < MAXM; ++m)
        if (m < M) {
          const float b = 1.f / y[m];
          P = fmaf(gs[m], xtf[(size_t)t * M + m] * b * b, P);
          Rr = fmaf(gs[m], b, Rr);
        }
      const float w = a.v[t] * a.R[(size_t)f * T + t];
      num = fmaf(w, P, num);
      den = fmaf(w, Rr, den);
    }
    const float2 s = block_sum2(num, den, red);
    if (tid == 0) {
      const float u = a.u[f] * sqrtf(s.x / s.y);
      if (!isfinite(u)) flag(a.p.status, ST_NONFINITE);
      a.u[f] = u;
      uf_s = u;
    }
    __syncthreads();
    const float u = uf_s;
    for (int t = tid; t < T; t += kThreads) a.lam[(size_t)f * T + t] = u * a.v[t] * a.R[(size_t)f * T + t];
    return;
  }
  // mode 1: the noise bases of the bin, one (n, k) pair per thread
  const int np = (N - 1) * K;
  float an = 0.f, ad = 0.f;
  for (int t0 = 0; t0 < T; t0 += kThreads) {
    const int t = t0 + tid;
    if (t < T) {
      float y[MAXM], A[MAXM], B[MAXM];
      bin_y<MAXM>(a.lam, gs, N, M, FT, (size_t)f * T + t, y);
#pragma unroll
      for (int m = 0; m < MAXM; ++m) {
        B[m] = (m < M) ? 1.f / y[m] : 0.f;
        A[m] = (m < M) ? xtf[(size_t)t * M + m] * B[m] * B[m] : 0.f;
      }
      for (int n = 1; n < N; ++n) {
        float P = 0.f, Rr = 0.f;
#pragma unroll
        for (int m = 0; m < MAXM; ++m)
          if (m < M) {
            P = fmaf(gs[n * MAXM + m], A[m], P);
            Rr = fmaf(gs[n * MAXM + m], B[m], Rr);
          }
        Ps[n - 1][tid] = P;
        Rs[n - 1][tid] = Rr;
      }
    }
    __syncthreads();
    if (tid < np) {
      const int n1 = tid / K;
      const float* hr = a.Hn + (size_t)tid * T + t0;
      const int tc = min(kThreads, T - t0);
      for (int j = 0; j < tc; ++j) {
        const float hv = hr[j];
        an = fmaf(hv, Ps[n1][j], an);
        ad = fmaf(hv, Rs[n1][j], ad);
      }
    }
    __syncthreads();
  }
  if (tid < np) {
    const size_t wi = (size_t)tid * F + f;
    const float w = a.Wn[wi] * sqrtf(an / ad);
    if (!isfinite(w)) flag(a.p.status, ST_NONFINITE);
    a.Wn[wi] = w;
    ws[tid] = w;
  }
  __syncthreads();
  for (int t = tid; t < T; t += kThreads)
    for (int n = 1; n < N; ++n) {
      float l = 0.f;
      for (int k = 0; k < K; ++k) l = fmaf(ws[(n - 1) * K + k], a.Hn[((size_t)(n - 1) * K + k) * T + t], l);
      a.lam[n * FT + (size_t)f * T + t] = l;
    }
}

// ---------------------------------------------------------------------------------------
// k_dp_tsweep: one CTA per kDpTT frames; thread (tl, fl) = (tid % 8, tid / 8) walks bins
// fl, fl + 32, ...
//  mode 0: v_t <- v_t sqrt( sum_f u_f r_tf P0_ft / sum_f u_f r_tf R0_ft ); lambda_ft0 anew;
//  mode 1: h_nkt <- h_nkt sqrt( sum_f w_nkf Pn_ft / sum_f w_nkf Rn_ft ) for n >= 1 (Eq. 24),
//          Pn, Rn of 32 bins staged in shared memory; lambda_ftn anew.
// ---------------------------------------------------------------------------------------
template <int MAXM>
__global__ void __launch_bounds__(kThreads) k_dp_tsweep(DpArgs a, int mode) {
  __shared__ float Ps[7][kDpFC][kDpTT], Rs[7][kDpFC][kDpTT];
  __shared__ float rn[kDpFC][kDpTT], rd[kDpFC][kDpTT];
  __shared__ float hs[kDpMaxPairs * kDpTT];
  __shared__ float vs[kDpTT];
  const int F = a.p.F, T = a.p.T, M = a.p.M, N = a.p.N, K = a.K;
  const size_t FT = (size_t)F * T;
  const int tid = threadIdx.x, tl = tid % kDpTT, fl = tid / kDpTT;
  const int t0 = blockIdx.x * kDpTT, t = t0 + tl;
  const bool valid = t < T;
  const int np = (N - 1) * K;
  float an[kDpItems], ad[kDpItems];
#pragma unroll
  for (int i = 0; i < kDpItems; ++i) an[i] = ad[i] = 0.f;
  float num = 0.f, den = 0.f;
  for (int f0 = 0; f0 < F; f0 += kDpFC) {
    const int f = f0 + fl;
    if (valid && f < F) {
      const float* gf = a.p.G + (size_t)f * M;  // g~_nfm at gf[n F M + m]
      const size_t gn = (size_t)F * M;
      float y[MAXM], A[MAXM], B[MAXM];
#pragma unroll
      for (int m = 0; m < MAXM; ++m) y[m] = 0.f;
      for (int n = 0; n < N; ++n) {
        const float l = a.lam[n * FT + (size_t)f * T + t];
#pragma unroll
        for (int m = 0; m < MAXM; ++m)
          if (m < M) y[m] = fmaf(l, gf[n * gn + m], y[m]);
      }
      const float* xp = a.p.xt + ((size_t)f * T + t) * M;
#pragma unroll
      for (int m = 0; m < MAXM; ++m) {
        B[m] = (m < M) ? 1.f / y[m] : 0.f;
        A[m] = (m < M) ? xp[m] * B[m] * B[m] : 0.f;
      }
      if (mode == 0) {
        float P = 0.f, Rr = 0.f;
#pragma unroll
        for (int m = 0; m < MAXM; ++m)
          if (m < M) {
            P = fmaf(gf[m], A[m], P);
            Rr = fmaf(gf[m], B[m], Rr);
          }
        const float w = a.u[f] * a.R[(size_t)f * T + t];
        num = fmaf(w, P, num);
        den = fmaf(w, Rr, den);
      } else {
        for (int n = 1; n < N; ++n) {
          float P = 0.f, Rr = 0.f;
#pragma unroll
          for (int m = 0; m < MAXM; ++m)
            if (m < M) {
              P = fmaf(gf[n * gn + m], A[m], P);
              Rr = fmaf(gf[n * gn + m], B[m], Rr);
            }
          Ps[n - 1][fl][tl] = P;
          Rs[n - 1][fl][tl] = Rr;
        }
      }
    } else if (mode == 1) {
      for (int n = 1; n < N; ++n) Ps[n - 1][fl][tl] = Rs[n - 1][fl][tl] = 0.f;
    }
    if (mode == 1) {
      __syncthreads();
      const int fc = min(kDpFC, F - f0);
#pragma unroll
      for (int i = 0; i < kDpItems; ++i) {
        const int item = tid + i * kThreads;
        if (item < np * kDpTT) {
          const int pair = item / kDpTT, tl2 = item - pair * kDpTT, n1 = pair / K;
          const float* wr = a.Wn + (size_t)pair * F + f0;
          for (int j = 0; j < fc; ++j) {
            const float w = wr[j];
            an[i] = fmaf(w, Ps[n1][j][tl2], an[i]);
            ad[i] = fmaf(w, Rs[n1][j][tl2], ad[i]);
          }
        }
      }
      __syncthreads();
    }
  }
  if (mode == 0) {
    rn[fl][tl] = num;
    rd[fl][tl] = den;
    __syncthreads();
    if (tid < kDpTT && t0 + tid < T) {
      float sn = 0.f, sd = 0.f;
      for (int j = 0; j < kDpFC; ++j) {
        sn += rn[j][tid];
        sd += rd[j][tid];
      }
      const float v = a.v[t0 + tid] * sqrtf(sn / sd);
      if (!isfinite(v)) flag(a.p.status, ST_NONFINITE);
      a.v[t0 + tid] = v;
      vs[tid] = v;
    }
    __syncthreads();
    if (valid)
      for (int f = fl; f < F; f += kDpFC) a.lam[(size_t)f * T + t] = a.u[f] * vs[tl] * a.R[(size_t)f * T + t];
    return;
  }
#pragma unroll
  for (int i = 0; i < kDpItems; ++i) {
    const int item = tid + i * kThreads;
    if (item < np * kDpTT) {
      const int pair = item / kDpTT, tl2 = item - pair * kDpTT;
      if (t0 + tl2 < T) {
        const size_t hi = (size_t)pair * T + t0 + tl2;
        const float hv = a.Hn[hi] * sqrtf(an[i] / ad[i]);
        if (!isfinite(hv)) flag(a.p.status, ST_NONFINITE);
        a.Hn[hi] = hv;
        hs[pair * kDpTT + tl2] = hv;
      }
    }
  }
  __syncthreads();
  if (valid)
    for (int f = fl; f < F; f += kDpFC)
      for (int n = 1; n < N; ++n) {
        float l = 0.f;
        for (int k = 0; k < K; ++k)
          l = fmaf(a.Wn[((size_t)(n - 1) * K + k) * F + f], hs[((n - 1) * K + k) * kDpTT + tl], l);
        a.lam[n * FT + (size_t)f * T + t] = l;
      }
}

// ---------------------------------------------------------------------------------------
// k_dp_norm: CTA 0 scales u_f by nu_0f, then mu_0 = sum_f u_f: u /= mu_0, v *= mu_0; CTA
// 1 + (n-1) K + k scales w_nkf by nu_nf, then mu_nk = sum_f w_nkf: w /= mu, h *= mu.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_dp_norm(DpArgs a) {
  __shared__ float red[2 * (kThreads / 32)];
  const int F = a.p.F, T = a.p.T;
  const int row = blockIdx.x;
  float* x = row == 0 ? a.u : a.Wn + (size_t)(row - 1) * F;
  float* y = row == 0 ? a.v : a.Hn + (size_t)(row - 1) * T;
  const float* nu = a.nu + (size_t)(row == 0 ? 0 : 1 + (row - 1) / a.K) * F;
  float s = 0.f;
  for (int f = threadIdx.x; f < F; f += kThreads) s += x[f] * nu[f];
  const float mu = block_sum2(s, 0.f, red).x;
  if (!(mu > 0.f) || !isfinite(mu)) flag(a.p.status, ST_NONFINITE);
  for (int f = threadIdx.x; f < F; f += kThreads) x[f] = x[f] * nu[f] / mu;
  for (int t = threadIdx.x; t < T; t += kThreads) y[t] *= mu;
}

}  // namespace

int dp_mh_frames(int F, int T, int M, int D, int Hd, int sms, size_t limit, size_t* smem) {
  // the most frames per CTA (each row of W2 read once serves them all) that still gives every
  // SM about 1.5 CTAs and fits the staging in shared memory
  for (int tb = 4; tb >= 1; tb >>= 1) {
    const size_t b = (size_t)mh_layout(F, M, tb, D, Hd).total * sizeof(float);
    if (b > limit) continue;
    if (tb > 1 && 2 * ((T + tb - 1) / tb) < 3 * sms) continue;
    if (smem) *smem = b;
    return tb;
  }
  return 0;
}

namespace {
template <int MAXM>
cudaError_t mh_prepare(size_t smem) {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_dp_mh<MAXM, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_dp_mh<MAXM, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_dp_mh<MAXM, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}
// Threads of a Metropolis CTA: whole warps, one bin per thread where F allows, the bins
// spread evenly over the rounds otherwise (no round for a few tail bins).
int mh_threads(int F) {
  const int rounds = (F + kMhMaxThreads - 1) / kMhMaxThreads;
  const int per = (F + rounds - 1) / rounds;
  return ((per + 31) / 32) * 32;
}
template <int MAXM>
cudaError_t mh_launch(const DpArgs& a, size_t smem, cudaStream_t st) {
  const dim3 grid((a.p.T + a.tb - 1) / a.tb);
  const int nthr = mh_threads(a.p.F);
  switch (a.tb) {
    case 4: k_dp_mh<MAXM, 4><<<grid, nthr, smem, st>>>(a); break;
    case 2: k_dp_mh<MAXM, 2><<<grid, nthr, smem, st>>>(a); break;
    default: k_dp_mh<MAXM, 1><<<grid, nthr, smem, st>>>(a); break;
  }
  return cudaGetLastError();
}
}  // namespace

cudaError_t dp_prepare(int maxm, size_t mh_smem) {
  switch (maxm) {
    case 2: return mh_prepare<2>(mh_smem);
    case 4: return mh_prepare<4>(mh_smem);
    default: return mh_prepare<8>(mh_smem);
  }
}

cudaError_t dp_launch_init(const DpArgs& a, cudaStream_t st) {
  constexpr int TB = 4;
  const size_t smem = (size_t)(TB * a.Hd + TB * a.D) * sizeof(float);
  k_dp_init<TB><<<(a.p.T + TB - 1) / TB, kThreads, smem, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || a.p.N < 2) return e;
  const size_t FT = (size_t)a.p.F * a.p.T;
  k_dp_lam_noise<<<(unsigned)((FT + kThreads - 1) / kThreads), kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t dp_launch_mh(const DpArgs& a, size_t smem, cudaStream_t st) {
  switch (a.maxm) {
    case 2: return mh_launch<2>(a, smem, st);
    case 4: return mh_launch<4>(a, smem, st);
    default: return mh_launch<8>(a, smem, st);
  }
}

cudaError_t dp_launch_fsweep(const DpArgs& a, int mode, cudaStream_t st) {
  switch (a.maxm) {
    case 2: k_dp_fsweep<2><<<a.p.F, kThreads, 0, st>>>(a, mode); break;
    case 4: k_dp_fsweep<4><<<a.p.F, kThreads, 0, st>>>(a, mode); break;
    default: k_dp_fsweep<8><<<a.p.F, kThreads, 0, st>>>(a, mode); break;
  }
  return cudaGetLastError();
}

cudaError_t dp_launch_tsweep(const DpArgs& a, int mode, cudaStream_t st) {
  const dim3 grid((a.p.T + kDpTT - 1) / kDpTT);
  switch (a.maxm) {
    case 2: k_dp_tsweep<2><<<grid, kThreads, 0, st>>>(a, mode); break;
    case 4: k_dp_tsweep<4><<<grid, kThreads, 0, st>>>(a, mode); break;
    default: k_dp_tsweep<8><<<grid, kThreads, 0, st>>>(a, mode); break;
  }
  return cudaGetLastError();
}

cudaError_t dp_launch_norm(const DpArgs& a, cudaStream_t st) {
  k_dp_norm<<<1 + (a.p.N - 1) * a.K, kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace fm
