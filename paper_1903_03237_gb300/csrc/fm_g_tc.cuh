// The g~ update (Eq. 21) on the tensor cores, mixed-precision form.
//
//   num_nfm = sum_t lambda_nft x~_ftm / y~_ftm^2,  den_nfm = sum_t lambda_nft / y~_ftm,
//   g~_nfm <- g~_nfm sqrt(num_nfm / den_nfm),      y~_ftm = sum_n lambda_nft g~_nfm (old g~)
//
// For one bin this is a [2M x T] . [T x N] contraction.  A CTA stacks FG = 64 / MAXM bins
// so that the A tile has 128 rows (ab, g, m) = (x~/y~^2 or 1/y~, bin, channel) and the B
// tile NC = FG * NP rows (g', n) of lambda (N padded to NP); of
//   D[(ab, g, m)][(g', n)] = sum_t A[(ab, g, m)][t] lambda_{f_g' n t}
// only the blocks g == g' are kept.  Operands are split BF16 (hi*hi + hi*lo + lo*hi, about
// 16 significant bits); a TMEM accumulator sums at most 256 frames, finished blocks are
// added into registers.
//
// The kernel follows the V_fm kernel's organisation: warps 0-3 form the operands and own
// the TMEM lanes, warp 4 issues the MMAs and the TMA tile copies of the x~ and lambda boxes
// (tensor maps; kGtcIn stages ahead, when T is a multiple of 4); they meet at mbarriers.
// Shared-memory layouts: x~ [bin][frame][channel], lambda [source][bin][frame].
// Per stage of 32 frames the threads form, per (bin, 8 frames, channel), y~ from lambda and
// g~ and the A rows x~/y~^2 and 1/y~, and per (bin, 8 frames, source) the lambda rows.
// Each split writes partial sums part[S][2][N][F][M]; the last CTA of a bin group to
// finish sums them in split order and applies the update.
#pragma once
#include <cuda.h>

#include "fm_common.cuh"
#include "fm_kernels.cuh"
#include "fm_tc.cuh"

namespace fm {

constexpr int kGtcThreads = 128;
constexpr int kGtcKc = 32;           // frames per stage (two BF16 MMA k-steps)
constexpr int kGtcBlockFrames = 256;
constexpr int kGtcIn = 2;            // input stages in flight (TMA runs up to 2 stages ahead)

template <int MAXM, int NP>
struct GtcCfg {
  static constexpr int FG = 64 / MAXM;           // bins per CTA
  static constexpr int NC = FG * NP;             // MMA N
  static constexpr int SPB = kGtcBlockFrames / kGtcKc;
  static constexpr int A_BYTES = 128 * kGtcKc * 2;
  static constexpr int B_BYTES = NC * kGtcKc * 2;
  static constexpr int OPS = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr int XT_BYTES = FG * kGtcKc * MAXM * 4;  // one stage of x~ rows
  static constexpr uint32_t TCOLS = 2 * NC < 32 ? 32 : 2 * NC;
  static constexpr int NFG = kGtcKc / 8;         // 8-frame groups per stage
  static constexpr int NA_ITEMS = FG * NFG * MAXM;  // A items (bin, frame group, channel)
  static constexpr int NB_ITEMS = FG * NFG * NP;    // lambda rows (bin, frame group, source)
  static_assert(NC >= 16 && NC <= 256 && NC % 16 == 0, "MMA N");
  static_assert((32 / MAXM) * NP % 16 == 0, "a warp reads whole 16-column groups of its bins");
  static_assert(FG * MAXM == 64, "A rows (ab, bin, channel) fill the 128 MMA rows");
  __host__ __device__ static int lam_bytes(int N) { return FG * N * kGtcKc * 4; }
  __host__ __device__ static int smem(int N) { return 2 * OPS + kGtcIn * (XT_BYTES + lam_bytes(N)) + FG * N * MAXM * 4; }
};

template <int MAXM, int NP>
__global__ void __launch_bounds__(kGtcThreads + 32, 4) k_g_tc(Prob p, int S, int span, unsigned ctr_base, int tma,
                                                              const __grid_constant__ CUtensorMap tm_xt,
                                                              const __grid_constant__ CUtensorMap tm_lam) {
  using C = GtcCfg<MAXM, NP>;
  constexpr int KC = kGtcKc;
  extern __shared__ __align__(1024) unsigned char ssm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ __align__(8) uint64_t xbar[kGtcIn];
  __shared__ __align__(8) uint64_t rbar[2];
  __shared__ __align__(8) uint64_t never_bar;  // nothing arrives here (test limit only)
  __shared__ int s_to, s_mma_last;             // a wait ran out; last stage with committed MMAs
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int F = p.F, T = p.T, N = p.N, M = p.M;
  const int f0 = blockIdx.x * C::FG;
  const int s = blockIdx.y;
  const int tbeg = s * span, tend = min(T, tbeg + span);
  const int nst = tend > tbeg ? (tend - tbeg + KC - 1) / KC : 0;
  const int nbins = min(C::FG, F - f0);
  // tma: the host encoded the tensor maps (T a multiple of 4, so that the row strides are
  // multiples of 16 bytes); otherwise the inputs are loaded by the threads
  const bool use_tma = tma != 0;
  const int IN_BYTES = C::XT_BYTES + C::lam_bytes(N);
  auto xbuf = [&](int c) { return reinterpret_cast<float*>(ssm + 2 * C::OPS + (c % kGtcIn) * IN_BYTES); };
  auto lbuf = [&](int c) { return reinterpret_cast<float*>(ssm + 2 * C::OPS + (c % kGtcIn) * IN_BYTES + C::XT_BYTES); };
  float* gs = reinterpret_cast<float*>(ssm + 2 * C::OPS + kGtcIn * IN_BYTES);  // g~ [FG][N][MAXM]
  constexpr int MMA_WARP = kGtcThreads / 32;

  if (warp == 0) { tmem_alloc(&tbase, C::TCOLS); tmem_relinquish(); }
  if (tid == 0) {
    mbar_init(&mbar[0], 1); mbar_init(&mbar[1], 1);
    for (int i = 0; i < kGtcIn; ++i) mbar_init(&xbar[i], 1);
    mbar_init(&rbar[0], kGtcThreads); mbar_init(&rbar[1], kGtcThreads);
    mbar_init(&never_bar, 1);
    s_to = 0;
    s_mma_last = -1;
  }
  for (int e = tid; e < C::FG * N * MAXM; e += kGtcThreads + 32) {
    const int g = e / (N * MAXM), r = e % (N * MAXM), n = r / MAXM, m = r % MAXM;
    gs[e] = (g < nbins && m < M) ? p.G[((size_t)n * F + f0 + g) * M + m] : 0.f;
  }
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tacc = tbase;
  constexpr uint32_t idesc = idesc_bf16_f32(128, C::NC);
  constexpr uint32_t kMaxTries = 1u << 22;
  const uint32_t lim = p.wait_limit ? p.wait_limit : kMaxTries;  // consumer waits
  bool ok = true;

  // register accumulators: TMEM lane r = A row (ab, g, m); columns g*NP + n
  const int r = tid;
  const int rab = r >> 6, rg = (r & 63) / MAXM, rm = r % MAXM;
  float vacc[NP];
#pragma unroll
  for (int n = 0; n < NP; ++n) vacc[n] = 0.f;

  if (warp == MMA_WARP) {
    // ------------------------------ input copies and MMAs ------------------------------
    // one tiled copy per array and stage: the x~ box (KC*M values of FG bins) and the lambda
    // box (KC frames x FG bins x N sources); zero fill past T and F
    auto issue_in = [&](int c) {
      const int t0 = tbeg + c * KC;
      if (lane == 0) {
        fence_async_smem();
        uint64_t* xb = &xbar[c % kGtcIn];
        mbar_expect_tx(xb, (uint32_t)(C::XT_BYTES / MAXM * M + C::lam_bytes(N)));
        tma_tile_2d(xbuf(c), &tm_xt, t0 * M, f0, xb);
        tma_tile_3d(lbuf(c), &tm_lam, t0, f0, 0, xb);
      }
      __syncwarp();
    };
    int issued = -1;
    if (use_tma) {
      for (int c = 0; c < min(kGtcIn, nst); ++c) issue_in(c);
      issued = min(kGtcIn, nst) - 1;
    }
    int mma_last = -1;
    for (int c = 0; c < nst; ++c) {
      uint64_t* wb = (p.wait_limit && c == 0) ? &never_bar : &rbar[c & 1];  // test limit: runs out
      // warp-uniform decision: the lanes meet at __syncwarp below
      if (!__all_sync(0xffffffffu, mbar_wait(wb, (uint32_t)((c >> 1) & 1), lim))) { ok = false; break; }
      tc_fence_after();
      mma_last = c;
      if (lane == 0) {
        unsigned char* st = ssm + (c & 1) * C::OPS;
        const uint32_t acc = tacc + (uint32_t)(((c / C::SPB) & 1) * C::NC);
        const uint32_t sah = smem_u32(st), sal = sah + C::A_BYTES;
        const uint32_t sbh = sah + 2 * C::A_BYTES, sbl = sbh + C::B_BYTES;
        constexpr uint32_t ALBO = 128 * 16, BLBO = C::NC * 16;
#pragma unroll
        for (int q = 0; q < KC / 16; ++q) {
          const uint64_t ah = umma_desc(sah + q * 2 * ALBO, ALBO, 128), al = umma_desc(sal + q * 2 * ALBO, ALBO, 128);
          const uint64_t bh = umma_desc(sbh + q * 2 * BLBO, BLBO, 128), bl = umma_desc(sbl + q * 2 * BLBO, BLBO, 128);
          umma_f16(acc, ah, bh, idesc, (c % C::SPB != 0 || q > 0) ? 1u : 0u);
          umma_f16(acc, ah, bl, idesc, 1u);
          umma_f16(acc, al, bh, idesc, 1u);
        }
        umma_commit(&mbar[c & 1]);
      }
      __syncwarp();
      // then the copies of stage c + kGtcIn into stage c's (consumed) input buffer: issuing
      // the MMAs first keeps them off the copies' issue time
      if (use_tma && c + kGtcIn < nst) { issue_in(c + kGtcIn); issued = c + kGtcIn; }
    }
    if (lane == 0) s_mma_last = mma_last;
    if (!ok) {
      if (lane == 0) { atomicOr(p.status, ST_TIMEOUT); s_to = 1; }
      // copies still in flight land before the CTA releases its shared memory (bounded)
      for (int c = max(0, issued - kGtcIn + 1); c <= issued; ++c)
        mbar_wait(&xbar[c % kGtcIn], (uint32_t)((c / kGtcIn) & 1), kMaxTries);
    }
  } else {
    // ------------------------------ operand formation ------------------------------
    // TMEM columns a warp reads: the bins of its 32 rows
    constexpr int BPW = 32 / MAXM;                 // bins per warp
    const int gw0 = ((32 * warp) & 63) / MAXM;     // first bin of this warp's rows
    auto flush = [&](int blk) {
      const uint32_t base = tacc + ((uint32_t)(32 * warp) << 16) + (uint32_t)((blk & 1) * C::NC + gw0 * NP);
#pragma unroll 1
      for (int cc = 0; cc < BPW * NP; cc += 16) {
        float v[16];
        tmem_ld16(base + (uint32_t)cc, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int rel = cc + j - (rg - gw0) * NP;  // column within this lane's bin
#pragma unroll
          for (int n = 0; n < NP; ++n)
            if (rel == n) vacc[n] += v[j];
        }
      }
    };
    int c = 0;
    for (; c < nst; ++c) {
      const int t0 = tbeg + c * KC, nt = min(KC, tend - t0);
      unsigned char* st = ssm + (c & 1) * C::OPS;
      unsigned char* Ah = st;
      unsigned char* Al = st + C::A_BYTES;
      unsigned char* Bh = st + 2 * C::A_BYTES;
      unsigned char* Bl = Bh + C::B_BYTES;
      // decisions are warp-uniform at least: flush() reads TMEM with a warp-collective load
      const bool to = c >= 2 && !__all_sync(0xffffffffu, mbar_wait(&mbar[c & 1], (uint32_t)(((c - 2) >> 1) & 1), lim));
      tc_fence_after();
      if (!to && c >= 2 && (c - 2) % C::SPB == C::SPB - 1) flush((c - 2) / C::SPB);
      float* xs = xbuf(c);
      float* ls = lbuf(c);
      if (use_tma) {
        // no barrier among the formation warps on this path: each may leave on its own
        if (to || !__all_sync(0xffffffffu, mbar_wait(&xbar[c % kGtcIn], (uint32_t)((c / kGtcIn) & 1), lim))) {
          ok = false;
          break;
        }
      } else {
        for (int e = tid; e < nbins * nt * M; e += kGtcThreads) {
          const int g = e / (nt * M), j = e - g * (nt * M);
          xs[g * KC * M + j] = p.xt[((size_t)(f0 + g) * T + t0) * M + j];
        }
        for (int e = tid; e < nbins * N * nt; e += kGtcThreads) {
          const int gn = e / nt, t = e - gn * nt, g = gn / N, n = gn % N;
          ls[(n * C::FG + g) * KC + t] = p.lam[((size_t)n * F + f0 + g) * T + t0 + t];
        }
        // barrier 1 over the formation warps, with the OR of their timeout flags: they leave
        // together
        uint32_t any;
        asm volatile(
            "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
            : "=r"(any)
            : "r"(to ? 1u : 0u), "n"(kGtcThreads)
            : "memory");
        if (any) { ok = false; break; }
      }
      // ---- A rows: x~/y~^2 and 1/y~ for 8 frames of (bin, channel); rows (ab, g, m) ----
      for (int e = tid; e < C::NA_ITEMS; e += kGtcThreads) {
        const int a_m = e % MAXM, a_g = (e / MAXM) % C::FG, a_fgrp = e / (MAXM * C::FG);
        const bool a_ok = (a_g < nbins) && (a_m < M);
        const int a_row = a_g * MAXM + a_m;
        const uint32_t a_off0 = (uint32_t)(a_fgrp * (128 * 16) + a_row * 16);
        const uint32_t a_off1 = a_off0 + 64 * 16;
        const int nv = min(8, nt - 8 * a_fgrp);
        float av[8], bv[8];
        if (a_ok && nv > 0) {
          float y[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) y[j] = 0.f;
          for (int n = 0; n < N; ++n) {
            const float gv = gs[(a_g * N + n) * MAXM + a_m];
            const float* lp = ls + (n * C::FG + a_g) * KC + 8 * a_fgrp;
            const float4 l0 = *reinterpret_cast<const float4*>(lp);
            const float4 l1 = *reinterpret_cast<const float4*>(lp + 4);
            y[0] = fmaf(l0.x, gv, y[0]); y[1] = fmaf(l0.y, gv, y[1]); y[2] = fmaf(l0.z, gv, y[2]); y[3] = fmaf(l0.w, gv, y[3]);
            y[4] = fmaf(l1.x, gv, y[4]); y[5] = fmaf(l1.y, gv, y[5]); y[6] = fmaf(l1.z, gv, y[6]); y[7] = fmaf(l1.w, gv, y[7]);
          }
          const float* xp = xs + (a_g * KC + 8 * a_fgrp) * M + a_m;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const bool v = j < nv;
            const float b = v ? __fdividef(1.f, y[j]) : 0.f;
            bv[j] = b;
            av[j] = v ? xp[j * M] * b * b : 0.f;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) { av[j] = 0.f; bv[j] = 0.f; }
        }
        uint4 hv, lv;
        split8(av, hv, lv);
        *reinterpret_cast<uint4*>(Ah + a_off0) = hv;
        *reinterpret_cast<uint4*>(Al + a_off0) = lv;
        split8(bv, hv, lv);
        *reinterpret_cast<uint4*>(Ah + a_off1) = hv;
        *reinterpret_cast<uint4*>(Al + a_off1) = lv;
      }
      // ---- B rows: lambda of 8 frames per (bin, source) ----
      for (int e = tid; e < C::NB_ITEMS; e += kGtcThreads) {
        const int n = e % NP, g = (e / NP) % C::FG, fgrp = e / (NP * C::FG);  // fgrp < NFG
        const int nv = min(8, nt - 8 * fgrp);
        float lv8[8];
        if (g < nbins && n < N && nv > 0) {
          const float* lp = ls + (n * C::FG + g) * KC + 8 * fgrp;
          const float4 l0 = *reinterpret_cast<const float4*>(lp);
          const float4 l1 = *reinterpret_cast<const float4*>(lp + 4);
          lv8[0] = l0.x; lv8[1] = l0.y; lv8[2] = l0.z; lv8[3] = l0.w;
          lv8[4] = l1.x; lv8[5] = l1.y; lv8[6] = l1.z; lv8[7] = l1.w;
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (j >= nv) lv8[j] = 0.f;
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) lv8[j] = 0.f;
        }
        uint4 hv, lo;
        split8(lv8, hv, lo);
        const uint32_t off = (uint32_t)(fgrp * (C::NC * 16) + (g * NP + n) * 16);
        *reinterpret_cast<uint4*>(Bh + off) = hv;
        *reinterpret_cast<uint4*>(Bl + off) = lo;
      }
      fence_async_smem();
      tc_fence_before();
      mbar_arrive(&rbar[c & 1]);
    }
    const int ndone = c;
    if (ok && ndone >= 1) {
      if (!__all_sync(0xffffffffu, mbar_wait(&mbar[(ndone - 1) & 1], (uint32_t)(((ndone - 1) >> 1) & 1), lim)))
        ok = false;
      tc_fence_after();
      if (ok) {
        const int last = (ndone - 1) / C::SPB;
        if (last >= 1 && ndone == last * C::SPB + 1) flush(last - 1);
        flush(last);
      }
    }
    if (!ok) {
      if (lane == 0) { atomicOr(p.status, ST_TIMEOUT); s_to = 1; }
    } else if (rg < nbins && rm < M) {
      // partials in the layout of the g~ sweep: part[s][(ab*N + n)*F + f][m]
      const size_t psz = (size_t)2 * N * F * M;
      float* part = p.part + (size_t)s * psz;
      const int f = f0 + rg;
#pragma unroll
      for (int n = 0; n < NP; ++n)
        if (n < N) part[((size_t)(rab * N + n) * F + f) * M + rm] = vacc[n];
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (s_to) {
    // after a timeout: the MMAs the MMA warp committed land before the TMEM is freed
    const int last = s_mma_last;
    if (tid == 0 && last >= 0) mbar_wait(&mbar[last & 1], (uint32_t)((last >> 1) & 1), kMaxTries);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  if (warp == 0) tmem_dealloc(tacc, C::TCOLS);

  // the last split of this bin group to finish applies g~ <- g~ sqrt(num / den)
  if (!arrive_last(p.counters + ctr_base + blockIdx.x, (unsigned)S)) return;
  const size_t psz = (size_t)2 * N * F * M;
  for (int e = tid; e < N * C::FG * M; e += kGtcThreads + 32) {
    const int m = e % M, g = (e / M) % C::FG, n = e / (M * C::FG);
    if (g >= nbins) continue;
    const size_t idx = ((size_t)n * F + f0 + g) * M + m;
    const float num = sum_splits(p.part + idx, psz, S);
    const float den = sum_splits(p.part + (size_t)N * F * M + idx, psz, S);
    const float v = p.G[idx] * sqrtf(num / den);
    if (!isfinite(v)) flag(p.status, ST_NONFINITE);
    p.G[idx] = v;
  }
}

}  // namespace fm
