// Weighted spatial covariances V_fm (Eq. 18) on the tensor cores, mixed-precision form.
//
// V_fm[q] = sum_t w_ftm p_q(x_ft),  w_ftm = 1 / y~_ftm,  p_q = the M^2 real products of
// x_ft x_ft^H (slot a*MAXM + c: Re(x_a conj x_c) for a <= c, Im(x_c conj x_a) for a > c).
// For one bin this is a [M^2 x T] . [T x M] contraction whose output is far smaller than
// any MMA tile, so a CTA stacks FG = 128 / MAXM^2 bins: the MMA computes
//   D[(g, q)][(g', m)] = sum_t p_q(x_{f_g t}) w_{f_g' t m}
// and only the diagonal blocks g == g' are kept (the tensor core does FG times the useful
// work, which costs nothing next to the CUDA-core product formation).
// Precision: split TF32.  Each operand value v is stored as hi = tf32(v) and
// lo = tf32(v - hi), and three MMAs accumulate hi*hi + hi*lo + lo*hi in FP32, about float32
// accuracy: single TF32 (or BF16) operands leave ~1e-3 relative errors in the IP update at
// M = 8, T = 4096, through the small off-diagonal entries of V_fm.
// Per chunk of 32 frames: the X rows of the FG bins arrive by TMA (cp.async.bulk with an
// mbarrier transaction count) when 16-byte aligned, by plain loads otherwise; the threads
// form y~ (from the materialised lambda and g~), write it (the state's y~ before the phi
// normalisation), and write the products and weights into the two K-major operand tiles;
// one thread issues the MMAs.  Split sums go to part[S][F][M][MAXM^2] for k_ip.
#pragma once
#include <cuda_bf16.h>

#include "fm_common.cuh"
#include "fm_tc.cuh"

namespace fm {

constexpr int kScmThreads = 128;
constexpr int kScmKc = 32;  // frames per chunk

template <int MAXM, bool TF32>
struct ScmCfg {
  static constexpr int MM = MAXM * MAXM;
  static constexpr int FG = 128 / MM;          // bins per CTA
  static constexpr int NC = FG * MAXM;         // MMA N (multiple of 16)
  static constexpr int ES = 4;                 // TF32 operands (hi and lo tiles)
  static constexpr int KB = kScmKc * ES;       // bytes per operand row per chunk
  static constexpr int A_BYTES = 128 * KB;
  static constexpr int B_BYTES = NC * KB;
  static constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;   // A_hi, A_lo, B_hi, B_lo
  static constexpr int X_BYTES = FG * kScmKc * MAXM * 8;   // staged X rows (complex64)
  static constexpr int SMEM = 2 * STAGE + X_BYTES;
  static constexpr uint32_t TCOLS = NC < 32 ? 32 : NC;
};

__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(mbar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(mbar))
      : "memory");
}

template <int MAXM, bool TF32>
__global__ void __launch_bounds__(kScmThreads) k_scm_tc(Prob p, int S, int span) {
  using C = ScmCfg<MAXM, TF32>;
  extern __shared__ __align__(1024) unsigned char ssm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ __align__(8) uint64_t xbar;
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int F = p.F, T = p.T, M = p.M, N = p.N;
  const int f0 = blockIdx.x * C::FG;
  const int s = blockIdx.y;
  const int tbeg = s * span, tend = min(T, tbeg + span);
  float2* xs = reinterpret_cast<float2*>(ssm + 2 * C::STAGE);
  // X rows of one bin are 16-byte aligned when T*M is even (the chunk offsets are 64*M*8)
  const bool tma_ok = ((T * M) & 1) == 0;

  if (warp == 0) { tmem_alloc(&tbase, C::TCOLS); tmem_relinquish(); }
  if (tid == 0) { mbar_init(&mbar[0], 1); mbar_init(&mbar[1], 1); mbar_init(&xbar, 1); }
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tacc = tbase;
  constexpr uint32_t idesc = idesc_tf32_f32(128, C::NC);
  constexpr uint32_t kMaxTries = 1u << 20;

  bool ok = true;
  int c = 0;
  for (int t0 = tbeg; t0 < tend; t0 += kScmKc, ++c) {
    const int nt = min(kScmKc, tend - t0);
    unsigned char* st = ssm + (c & 1) * C::STAGE;
    if (c >= 2 && !mbar_wait(&mbar[c & 1], (uint32_t)(((c - 2) >> 1) & 1), kMaxTries)) { ok = false; break; }
    // ---- X rows of the FG bins for frames [t0, t0 + nt) ----
    const uint32_t row_bytes = (uint32_t)nt * M * 8;
    const bool use_tma = tma_ok && (row_bytes % 16 == 0);
    if (use_tma) {
      if (tid == 0) {
        int nb = 0;
        for (int g = 0; g < C::FG; ++g) nb += (f0 + g < F);
        mbar_expect_tx(&xbar, row_bytes * (uint32_t)nb);
        for (int g = 0; g < C::FG; ++g)
          if (f0 + g < F) tma_bulk_g2s(xs + g * kScmKc * MAXM, p.X + ((size_t)(f0 + g) * T + t0) * M, row_bytes, &xbar);
      }
      if (!mbar_wait(&xbar, (uint32_t)(c & 1), kMaxTries)) { ok = false; break; }
    } else {
      for (int e = tid; e < C::FG * nt * M; e += kScmThreads) {
        const int g = e / (nt * M), j = e % (nt * M);
        if (f0 + g < F) xs[g * kScmKc * MAXM + j] = p.X[((size_t)(f0 + g) * T + t0) * M + j];
      }
      __syncthreads();
      if (tid == 0) {  // keep the transaction barrier's phase in step with the chunk index
        mbar_expect_tx(&xbar, 0);
      }
      if (!mbar_wait(&xbar, (uint32_t)(c & 1), kMaxTries)) { ok = false; break; }
    }
    // ---- operands: products (A) and weights (B), plus y~ ----
    for (int e = tid; e < C::FG * kScmKc; e += kScmThreads) {
      const int g = e / kScmKc, t = e % kScmKc;
      const int f = f0 + g;
      const bool v = (f < F) && (t < nt);
      float2 x[MAXM];
      float w[MAXM];
#pragma unroll
      for (int j = 0; j < MAXM; ++j) { x[j] = make_float2(0.f, 0.f); w[j] = 0.f; }
      if (v) {
#pragma unroll
        for (int j = 0; j < MAXM; ++j)
          if (j < M) x[j] = xs[g * kScmKc * MAXM + t * M + j];
        float y[MAXM];
#pragma unroll
        for (int m = 0; m < MAXM; ++m) y[m] = 0.f;
        for (int n = 0; n < N; ++n) {
          const float l = __ldg(p.lam + ((size_t)n * F + f) * T + t0 + t);
          const float* gp = p.G + ((size_t)n * F + f) * M;
#pragma unroll
          for (int m = 0; m < MAXM; ++m)
            if (m < M) y[m] = fmaf(l, __ldg(gp + m), y[m]);
        }
        const size_t pt = (size_t)f * T + t0 + t;
#pragma unroll
        for (int m = 0; m < MAXM; ++m)
          if (m < M) { p.yt[pt * M + m] = y[m]; w[m] = __fdividef(1.f, y[m]); }
      }
      unsigned char* Ah = st;
      unsigned char* Al = st + C::A_BYTES;
      unsigned char* Bh = st + 2 * C::A_BYTES;
      unsigned char* Bl = Bh + C::B_BYTES;
#pragma unroll
      for (int a = 0; a < MAXM; ++a)
#pragma unroll
        for (int cc = 0; cc < MAXM; ++cc) {
          const float pr = (a <= cc) ? (x[a].x * x[cc].x + x[a].y * x[cc].y) : (x[cc].y * x[a].x - x[cc].x * x[a].y);
          const uint32_t off = cm_offset(g * C::MM + a * MAXM + cc, t, C::KB, 4);
          const float hi = to_tf32(pr);
          *reinterpret_cast<float*>(Ah + off) = hi;
          *reinterpret_cast<float*>(Al + off) = to_tf32(pr - hi);
        }
#pragma unroll
      for (int m = 0; m < MAXM; ++m) {
        const uint32_t off = cm_offset(g * MAXM + m, t, C::KB, 4);
        const float hi = to_tf32(w[m]);
        *reinterpret_cast<float*>(Bh + off) = hi;
        *reinterpret_cast<float*>(Bl + off) = to_tf32(w[m] - hi);
      }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();  // operands complete; X rows consumed
    tc_fence_after();
    if (tid == 0) {
      const uint32_t sah = smem_u32(st), sal = sah + C::A_BYTES;
      const uint32_t sbh = sah + 2 * C::A_BYTES, sbl = sbh + C::B_BYTES;
      constexpr uint32_t SBO = (C::KB / 16) * 128;
#pragma unroll
      for (int q = 0; q < C::KB / 32; ++q) {
        const uint32_t o = q * 2 * 128;
        const uint64_t ah = umma_desc(sah + o, 128, SBO), al = umma_desc(sal + o, 128, SBO);
        const uint64_t bh = umma_desc(sbh + o, 128, SBO), bl = umma_desc(sbl + o, 128, SBO);
        umma_tf32(tacc, ah, bh, idesc, (c > 0 || q > 0) ? 1u : 0u);
        umma_tf32(tacc, ah, bl, idesc, 1u);
        umma_tf32(tacc, al, bh, idesc, 1u);
      }
      umma_commit(&mbar[c & 1]);
    }
  }
  const int nch = c;
  if (ok && nch >= 2 && !mbar_wait(&mbar[(nch - 2) & 1], (uint32_t)(((nch - 2) >> 1) & 1), kMaxTries)) ok = false;
  if (ok && nch >= 1 && !mbar_wait(&mbar[(nch - 1) & 1], (uint32_t)(((nch - 1) >> 1) & 1), kMaxTries)) ok = false;
  tc_fence_after();
  if (!ok) {
    if (lane == 0) atomicOr(p.status, ST_TIMEOUT);
  } else {
    // row r = (g, q) of D: keep the columns (g, m), m < M
    const int r = 32 * warp + lane;
    const int g = r / C::MM, q = r % C::MM;
    const int f = f0 + g;
    float* part = p.part + (size_t)s * F * M * C::MM;
#pragma unroll
    for (int cc = 0; cc < C::NC; cc += 16) {
      float v[16];
      tmem_ld16(tacc + ((uint32_t)(32 * warp) << 16) + (uint32_t)cc, v);
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        const int col = cc + jj, gg = col / MAXM, m = col % MAXM;
        if (gg == g && m < M && f < F) part[((size_t)f * M + m) * C::MM + q] = (nch > 0) ? v[jj] : 0.f;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tacc, C::TCOLS);
}

}  // namespace fm
