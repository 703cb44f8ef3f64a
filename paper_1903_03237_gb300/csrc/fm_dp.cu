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
#include <algorithm>

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "fm_launch.h"

namespace cg = cooperative_groups;

namespace fm {
namespace {

constexpr int kDpTT = 2;                  // frames per CTA of the per-frame sweeps
constexpr int kDpFC = kThreads / kDpTT;   // bins per chunk of the per-frame sweeps (128)
constexpr int kDpMaxPairs = 256;          // (N-1) K noise bases per sweep CTA
constexpr int kDpItems = kDpMaxPairs * kDpTT / kThreads;  // H-sweep items per thread (2)
constexpr int kMhMaxThreads = 320;       // threads of a Metropolis CTA (at most; two CTAs per SM)
constexpr int kMhMaxTB = 16;             // frames of a Metropolis cluster (at most)
constexpr int kMhMaxC = 8;               // CTAs of a Metropolis cluster (the portable limit)


// Shared-memory layout (floats) of one Metropolis CTA: FC bins of the cluster's split, TB
// frames, a cluster of C CTAs.  W2 rows are padded by 4 floats so that the float4 reads of
// consecutive bins fall on distinct banks.
struct MhLayout {
  int w2, b2, xs, yr, g0, uf, rold, rnew, h, zs, zn, vs, pl, pg, total;
};
__host__ __device__ inline MhLayout mh_layout(int FC, int M, int TB, int D, int Hd, int C) {
  MhLayout L;
  int o = 0;
  auto take = [&](int n) { const int at = o; o += (n + 3) & ~3; return at; };
  L.w2 = take(FC * (Hd + 4));  // W2 rows of the CTA's bins
  L.b2 = take(FC);
  L.xs = take(TB * M * FC);    // x~ [tb*M + m][fl]
  L.yr = take(TB * M * FC);    // y~^{-0} [tb*M + m][fl]
  L.g0 = take(M * FC);         // g~_0 [m][fl]
  L.uf = take(FC);             // u_f
  L.rold = take(TB * FC);      // r of the current z [tb][fl]
  L.rnew = take(TB * FC);      // r of the proposal
  L.h = take(TB * Hd);         // hidden layer [tb][j]
  L.zs = take(TB * D);         // z [tb][d]
  L.zn = take(TB * D);         // proposal
  L.vs = take(TB);             // v_t
  L.pl = take(TB * FC);        // log gamma terms summed per bin [tb][fl]
  L.pg = take(2 * C * TB);     // the cluster's partial sums [proposal parity][rank][tb]
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
// k_dp_mh: S Metropolis proposals for each of a cluster's TB frames (Sec. III-B-3).  With
// y~^{-0}_ftm = sum_{n>=1} lambda_ftn g~_nfm fixed, the log acceptance ratio of frame t is
//   log gamma_t = sum_{f,m} [ x~ (y_new - y_old) / (y_new y_old) - log(y_new / y_old) ],
//   y_old = lambda_old g~_0 + y~^{-0},  y_new = y_old + (lambda_new - lambda_old) g~_0,
// the change of Eq. 17 when lambda_ft0 alone changes (each term formed from the difference,
// so nothing cancels between two large sums).  Accepted where log u < log gamma_t.
//
// The C CTAs of a cluster split the bins (FC each) and keep their rows of the decoder's
// output layer W2 in shared memory for the whole launch, so W2 is read from L2 once per CTA
// rather than once per proposal.  Per proposal, each CTA computes 1/C of the hidden units of
// every frame and stores them into every CTA of the cluster (distributed shared memory);
// after a cluster barrier each thread decodes FG frames of one bin and forms their terms.
// Every CTA then sums its bins' terms per frame (a warp per frame, fixed order) and stores the
// sum into every CTA of the cluster (buffers alternating with the proposal's parity); after a
// second cluster barrier all CTAs add the C partial sums in rank order, so they all take the
// same decisions, and each updates its own bins.
// ---------------------------------------------------------------------------------------
template <int MAXM, int FG>
__global__ void __launch_bounds__(kMhMaxThreads, 2) k_dp_mh(DpArgs a) {
  extern __shared__ __align__(16) float dsm[];
  __shared__ int acc_s[kMhMaxTB];
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
  const int F = a.p.F, T = a.p.T, M = a.p.M, N = a.p.N, D = a.D, Hd = a.Hd, TB = a.tb;
  const int HdP = Hd + 4;
  const size_t FT = (size_t)F * T;
  const int tid = threadIdx.x, nthr = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = nthr >> 5;
  const int FC = (F + C - 1) / C, f0 = rank * FC, nfc = max(0, min(FC, F - f0));
  const int t0 = (blockIdx.x / C) * TB, nt = min(TB, T - t0);
  const MhLayout L = mh_layout(FC, M, TB, D, Hd, C);
  float* w2 = dsm + L.w2;
  float* b2 = dsm + L.b2;
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
  float* pl = dsm + L.pl;
  float* pg = dsm + L.pg;

  // ---- stage the CTA's bins (W2 rows, b2, g~_0, u) and the frames' x~, y~^{-0}, r, z
  for (int e = tid; e < nfc * (Hd >> 2); e += nthr) {
    const int fl = e / (Hd >> 2), j4 = e - fl * (Hd >> 2);
    reinterpret_cast<float4*>(w2 + fl * HdP)[j4] =
        __ldg(reinterpret_cast<const float4*>(a.W2 + (size_t)(f0 + fl) * Hd) + j4);
  }
  const int run = nt * M;  // x~ of the tile's frames is contiguous per bin
  for (int e = tid; e < nfc * run; e += nthr) {
    const int fl = e / run, r = e - fl * run, tb = r / M, m = r - tb * M;
    const size_t ft = (size_t)(f0 + fl) * T + t0 + tb;
    xs[(tb * M + m) * FC + fl] = a.p.xt[ft * M + m];
    float y = 0.f;
    for (int n = 1; n < N; ++n) y = fmaf(a.lam[n * FT + ft], a.p.G[((size_t)n * F + f0 + fl) * M + m], y);
    yr[(tb * M + m) * FC + fl] = y;
  }
  for (int e = tid; e < nfc * M; e += nthr) {
    const int fl = e / M, m = e - fl * M;
    g0[m * FC + fl] = a.p.G[(size_t)(f0 + fl) * M + m];
  }
  for (int fl = tid; fl < nfc; fl += nthr) {
    b2[fl] = a.b2[f0 + fl];
    uf[fl] = a.u[f0 + fl];
    for (int tb = 0; tb < nt; ++tb) rold[tb * FC + fl] = a.R[(size_t)(f0 + fl) * T + t0 + tb];
  }
  for (int e = tid; e < TB * Hd; e += nthr) h[e] = 0.f;  // rows of absent frames stay 0
  for (int e = tid; e < nt * D; e += nthr) zs[e] = a.Z[(size_t)t0 * D + e];
  if (tid < nt) vs[tid] = a.v[t0 + tid];
  unsigned n_acc = 0;
  // every CTA of the cluster has started and initialised its shared memory before any CTA
  // stores into another's
  cluster.sync();

  // this thread's bin and frames: item = g FC + fl, frames g FG .. g FG + FG - 1
  const int NG = TB / FG;
  const int g = tid / FC, fl = tid - g * FC;
  const bool own = g < NG && fl < nfc;
  const int JC = (Hd + C - 1) / C, j0 = rank * JC, nj = max(0, min(JC, Hd - j0));
  for (int s = 0; s < a.S; ++s) {
    // proposal z' = z + sqrt(eps) xi (every CTA of the cluster forms the same)
    const float* xi = a.xi + ((size_t)s * T + t0) * D;
    for (int e = tid; e < nt * D; e += nthr) zn[e] = fmaf(a.sqrt_eps, xi[e], zs[e]);
    __syncthreads();
    // this CTA's share of the hidden units, into every CTA of the cluster
    for (int e = tid; e < nt * nj; e += nthr) {
      const int tb = e / nj, j = j0 + (e - tb * nj);
      float v = a.b1[j];
      const float* w = a.W1 + (size_t)j * D;
      for (int d = 0; d < D; ++d) v = fmaf(w[d], zn[tb * D + d], v);
      v = tanhf(v);
      for (int c = 0; c < C; ++c) cluster.map_shared_rank(h, c)[tb * Hd + j] = v;
    }
    cluster.sync();
    if (own) {
      float sv[FG];
#pragma unroll
      for (int i = 0; i < FG; ++i) sv[i] = 0.f;
      const float4* w = reinterpret_cast<const float4*>(w2 + fl * HdP);
      const float* hg = h + g * FG * Hd;
#pragma unroll 2
      for (int j4 = 0; j4 < (Hd >> 2); ++j4) {
        const float4 wv = w[j4];
#pragma unroll
        for (int i = 0; i < FG; ++i) {
          const float4 hv = *reinterpret_cast<const float4*>(hg + i * Hd + 4 * j4);
          sv[i] = fmaf(wv.x, hv.x, sv[i]);
          sv[i] = fmaf(wv.y, hv.y, sv[i]);
          sv[i] = fmaf(wv.z, hv.z, sv[i]);
          sv[i] = fmaf(wv.w, hv.w, sv[i]);
        }
      }
      const float u = uf[fl], bias = b2[fl];
#pragma unroll
      for (int i = 0; i < FG; ++i) {
        const int tb = g * FG + i;
        if (tb < nt) {
          const float rn = expf(sv[i] + bias);
          rnew[tb * FC + fl] = rn;
          const float lo = u * vs[tb] * rold[tb * FC + fl];
          const float dl = u * vs[tb] * rn - lo;
          float acc = 0.f;
#pragma unroll
          for (int m = 0; m < MAXM; ++m)
            if (m < M) {
              const float gm = g0[m * FC + fl];
              const float yo = fmaf(lo, gm, yr[(tb * M + m) * FC + fl]);
              const float d = dl * gm;
              const float yn = yo + d;
              acc += xs[(tb * M + m) * FC + fl] * d / (yn * yo) - log1pf(d / yo);
            }
          pl[tb * FC + fl] = acc;
        }
      }
    }
    __syncthreads();
    // this CTA's sum per frame (a warp per frame, bins in a fixed order), into every CTA
    float* buf = pg + (s & 1) * C * TB;
    for (int tb = warp; tb < nt; tb += nw) {
      float cp = 0.f;
      for (int b = lane; b < nfc; b += 32) cp += pl[tb * FC + b];
      for (int o = 16; o > 0; o >>= 1) cp += __shfl_xor_sync(0xffffffffu, cp, o);
      if (lane < C) cluster.map_shared_rank(buf, lane)[rank * TB + tb] = cp;
    }
    cluster.sync();
    if (tid < nt) {
      float lg = 0.f;
      for (int c = 0; c < C; ++c) lg += buf[c * TB + tid];
      const int acc = a.logu[(size_t)s * T + t0 + tid] < lg;
      acc_s[tid] = acc;
      if (rank == 0) {
        n_acc += acc;
        if (a.loggamma) a.loggamma[(size_t)s * T + t0 + tid] = lg;
        if (isnan(lg)) flag(a.p.status, ST_NONFINITE);
      }
    }
    __syncthreads();
    // accepted frames take the proposal (each thread copies what it wrote or will read)
    for (int e = tid; e < nt * D; e += nthr)
      if (acc_s[e / D]) zs[e] = zn[e];
    if (own)
#pragma unroll
      for (int i = 0; i < FG; ++i) {
        const int tb = g * FG + i;
        if (tb < nt && acc_s[tb]) rold[tb * FC + fl] = rnew[tb * FC + fl];
      }
  }
  __syncthreads();

  // ---- the sampled z (rank 0), r and lambda_ft0 of the CTA's bins
  if (rank == 0)
    for (int e = tid; e < nt * D; e += nthr) a.Z[(size_t)t0 * D + e] = zs[e];
  for (int e = tid; e < nfc * nt; e += nthr) {
    const int b = e / nt, tb = e - b * nt;
    const size_t i = (size_t)(f0 + b) * T + t0 + tb;
    const float r = rold[tb * FC + b];
    a.R[i] = r;
    a.lam[i] = uf[b] * vs[tb] * r;
  }
  if (rank == 0 && tid < nt && n_acc) atomicAdd(a.n_acc, (unsigned long long)n_acc);
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
  __shared__ float sn_s[kThreads], sd_s[kThreads];  // slice sums of the noise W rule
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
  // mode 1: the noise bases of the bin; each (n, k) pair summed by nsl threads, each over every
  // nsl-th frame of a chunk, the slices added in order at the end
  const int np = (N - 1) * K;
  const int nsl = max(1, kThreads / np);
  const int pair = tid % np, sl = tid / np;
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
    if (sl < nsl) {
      const int n1 = pair / K;
      const float* hr = a.Hn + (size_t)pair * T + t0;
      const int tc = min(kThreads, T - t0);
#pragma unroll 8
      for (int j = sl; j < tc; j += nsl) {
        const float hv = hr[j];
        an = fmaf(hv, Ps[n1][j], an);
        ad = fmaf(hv, Rs[n1][j], ad);
      }
    }
    __syncthreads();
  }
  if (nsl > 1) {
    sn_s[tid] = an;
    sd_s[tid] = ad;
    __syncthreads();
    if (tid < np) {
      an = ad = 0.f;
      for (int q = 0; q < nsl; ++q) {
        an += sn_s[q * np + tid];
        ad += sd_s[q * np + tid];
      }
    }
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
  __shared__ float sn_s[kThreads], sd_s[kThreads];  // slice sums of the noise H rule
  __shared__ float vs[kDpTT];
  const int F = a.p.F, T = a.p.T, M = a.p.M, N = a.p.N, K = a.K;
  const size_t FT = (size_t)F * T;
  const int tid = threadIdx.x, tl = tid % kDpTT, fl = tid / kDpTT;
  const int t0 = blockIdx.x * kDpTT, t = t0 + tl;
  const bool valid = t < T;
  const int np = (N - 1) * K;
  const int nitems = np * kDpTT;                        // (pair, frame) items of the H rule
  const int nsl = (nitems > 0 && nitems < kThreads) ? kThreads / nitems : 1;  // threads per item
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
      if (nsl > 1) {
        // each (pair, frame) item summed by nsl threads over every nsl-th bin of the chunk
        if (tid < nsl * nitems) {
          const int item = tid % nitems, sl = tid / nitems;
          const int pair = item / kDpTT, tl2 = item - pair * kDpTT, n1 = pair / K;
          const float* wr = a.Wn + (size_t)pair * F + f0;
#pragma unroll 8
          for (int j = sl; j < fc; j += nsl) {
            const float w = wr[j];
            an[0] = fmaf(w, Ps[n1][j][tl2], an[0]);
            ad[0] = fmaf(w, Rs[n1][j][tl2], ad[0]);
          }
        }
      } else
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
  if (nsl > 1) {
    // the slices of each item added in order
    sn_s[tid] = an[0];
    sd_s[tid] = ad[0];
    __syncthreads();
    if (tid < nitems) {
      an[0] = ad[0] = 0.f;
      for (int q = 0; q < nsl; ++q) {
        an[0] += sn_s[q * nitems + tid];
        ad[0] += sd_s[q * nitems + tid];
      }
    }
  }
#pragma unroll
  for (int i = 0; i < kDpItems; ++i) {
    const int item = tid + i * kThreads;
    if (item < nitems) {
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

DpMhPlan dp_mh_plan(int F, int T, int M, int D, int Hd, int sms, size_t limit) {
  // about 64 bins per CTA; then the most frames per cluster (every W2 row read from shared
  // memory serves them all) that still puts a CTA on every SM and fits the staging
  DpMhPlan pl;
  const int C = std::min(kMhMaxC, std::max(1, (F + 63) / 64));
  const int FC = (F + C - 1) / C;
  for (int TB = kMhMaxTB; TB >= 1; TB >>= 1) {
    const size_t b = (size_t)mh_layout(FC, M, TB, D, Hd, C).total * sizeof(float);
    if (b > limit) continue;
    if (TB > 1 && ((T + TB - 1) / TB) * C < sms) continue;
    const int FG = std::min(TB, 4);
    const int thr = std::max(64, ((TB / FG * FC + 31) / 32) * 32);
    if (thr > kMhMaxThreads) continue;
    pl.C = C; pl.TB = TB; pl.FG = FG; pl.threads = thr; pl.smem = b;
    return pl;
  }
  return pl;
}

namespace {
template <int MAXM>
cudaError_t mh_prepare(size_t smem) {
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_dp_mh<MAXM, 1>, A, (int)smem)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_dp_mh<MAXM, 2>, A, (int)smem)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_dp_mh<MAXM, 4>, A, (int)smem);
}
template <int MAXM>
cudaError_t mh_launch(const DpArgs& a, const DpMhPlan& pl, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(((a.p.T + pl.TB - 1) / pl.TB) * pl.C);
  cfg.blockDim = dim3(pl.threads);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)pl.C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  switch (pl.FG) {
    case 4: return cudaLaunchKernelEx(&cfg, k_dp_mh<MAXM, 4>, a);
    case 2: return cudaLaunchKernelEx(&cfg, k_dp_mh<MAXM, 2>, a);
    default: return cudaLaunchKernelEx(&cfg, k_dp_mh<MAXM, 1>, a);
  }
}
}  // namespace

cudaError_t dp_prepare(int maxm, const DpMhPlan& pl) {
  switch (maxm) {
    case 2: return mh_prepare<2>(pl.smem);
    case 4: return mh_prepare<4>(pl.smem);
    default: return mh_prepare<8>(pl.smem);
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

cudaError_t dp_launch_mh(const DpArgs& a, const DpMhPlan& pl, cudaStream_t st) {
  switch (a.maxm) {
    case 2: return mh_launch<2>(a, pl, st);
    case 4: return mh_launch<4>(a, pl, st);
    default: return mh_launch<8>(a, pl, st);
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
