// Weighted spatial covariances V_fm (Eq. 18) on the tensor cores, mixed-precision form.
//
// V_fm[q] = sum_t w_ftm p_q(x_ft),  w_ftm = 1 / y~_ftm,  p_q = the M^2 real products of
// x_ft x_ft^H (q = a*MAXM + c: Re(x_a conj x_c) for a <= c, Im(x_c conj x_a) for a > c).
// For one bin this is a [M^2 x T] . [T x M] contraction whose output is far smaller than
// an MMA tile, so a CTA stacks FG = 128 / MAXM^2 bins: the MMA computes
//   D[(g, q)][(g', m)] = sum_t p_q(x_{f_g t}) w_{f_g' t m}
// and only the diagonal blocks g == g' are kept.
//
// Precision: split BF16.  Each operand value v is held as hi = bf16(v), lo = bf16(v - hi)
// (16 significant bits together) and three MMAs accumulate hi*hi + hi*lo + lo*hi in FP32.
// A single BF16 or TF32 product leaves ~1e-3 relative errors in the IP update at M = 8
// through the small off-diagonal entries of V_fm; the split brings them to ~1e-5.
// A TMEM accumulator sums at most 256 frames (bounding the growth of its sequential FP32
// rounding); two accumulators alternate and finished blocks are added into registers.
//
// Per stage of KC frames (KC = 32 for MAXM 8 and 4, 16 for MAXM 2: 128 product items):
//   - the X rows (per 8-frame group, into groups padded by 16 bytes so that the lanes'
//     loads spread over the banks) and lambda rows of the FG bins arrive by TMA
//     (cp.async.bulk with an mbarrier transaction count, issued by the lanes of warp 4; the
//     lambda rows as one tiled copy through a tensor map when the host made one)
//     IN stages ahead, when 16-byte aligned (T*M even, T a multiple of 4), else by plain
//     loads;
//   - y~ = sum_n lambda g~ for 8 frames per (bin, channel): written to the state (before
//     the phi normalisation) and, as 1/y~, into the B operand (one 16-byte row each);
//   - the products into the A operand: a thread owns (bin, c, 8 frames, a range), holds
//     x_c and sweeps a, storing one 16-byte core-matrix row (8 frames) per (a, hi/lo);
//   - one thread of a fifth warp issues KC/16 k-steps x 3 MMAs (M 128, N FG*MAXM, K 16)
//     and commits them; the same warp issues the input copies.
// Operand tiles use the K-major core-matrix layout with the 8-frame groups outermost
// (leading byte offset = rows * 16, stride byte offset = 128), which makes the 16-byte
// stores of 8 consecutive rows fill all 32 banks.  Rows of the A tile are ordered so that
// each 8-row group holds 8 distinct (bin, c): row = gq*8*MAXM + a*8 + gl*MAXM + c with
// g = gq*GL + gl, GL = 8 / MAXM.
// Split sums go to part[S][F][M][MAXM^2] for k_ip.
#pragma once
#include <cuda.h>

#include "fm_common.cuh"
#include "fm_tc.cuh"

namespace fm {

constexpr int kScmThreads = 128;
constexpr int kScmBlockFrames = 256;  // frames summed per TMEM accumulator
constexpr int kScmLamMax = 16384;     // lambda stage bytes above which lambda is read directly

template <int MAXM>
struct ScmCfg {
  static constexpr int MM = MAXM * MAXM;
  static constexpr int FG = 128 / MM;               // bins per CTA
  static constexpr int GL = 8 / MAXM;               // bins interleaved in one 8-row group
  static constexpr int NC = FG * MAXM;              // MMA N
  static constexpr int KC = (MAXM == 2) ? 16 : 32;  // frames per stage
  static constexpr int NFG = KC / 8;                // 8-frame groups per stage
  static constexpr int AP = 8 * MAXM / KC;          // a-ranges per (bin, c, frame group)
  static constexpr int SPB = kScmBlockFrames / KC;  // stages per accumulator block
  static constexpr int A_BYTES = 128 * KC * 2;      // one BF16 operand tile
  static constexpr int B_BYTES = NC * KC * 2;
  static constexpr int OPS = 2 * A_BYTES + 2 * B_BYTES;   // A hi, A lo, B hi, B lo
  // X rows staged per 8-frame group, groups padded by 16 bytes (bank spread):
  // group stride GS(M) = 8*M + 2 complex values
  static constexpr int X_BYTES = FG * NFG * (8 * MAXM + 2) * 8;
  static constexpr uint32_t TCOLS = 2 * NC < 32 ? 32 : 2 * NC;  // two accumulators
  static constexpr int NCW = (MAXM == 2) ? 16 : 8;       // accumulator columns a warp reads
  // input stages in flight: TMA runs up to IN stages ahead (3 where the stage inputs are
  // largest and the shared memory allows four CTAs per SM, else 2)
  static constexpr int IN = (MAXM == 8) ? 3 : 2;
  static constexpr int NB_ITEMS = FG * MAXM * NFG;       // weight items (bin, m, 8 frames)
  static_assert(FG * MAXM * NFG * AP == kScmThreads, "one product item per thread");
  static_assert(kScmThreads % NB_ITEMS == 0, "weight items spread evenly over the threads");
  // lambda stage bytes (0 when lambda is read directly) and total dynamic shared memory
  __host__ __device__ static int lam_bytes(int N) {
    const int b = FG * N * KC * 4;
    return b <= kScmLamMax ? b : 0;
  }
  __host__ __device__ static int smem(int N) {
    return 2 * OPS + IN * (X_BYTES + lam_bytes(N)) + FG * N * MAXM * 4;
  }
};

// Products of 8 frames of one (bin, c) with x_a for the a-range [a0, a0 + AR): hi and lo
// rows into the A tiles.  FULL: all 8 frames valid (no per-frame test).
template <int MAXM, int AR, bool FULL>
__device__ __forceinline__ void form_products(const float2* __restrict__ xg, int M, int nv, int cc, int a0,
                                              unsigned char* Ah, unsigned char* Al, uint32_t obase, int arow0) {
  float2 xc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) xc[j] = (FULL || j < nv) ? xg[j * M + cc] : make_float2(0.f, 0.f);
#pragma unroll
  for (int ai = 0; ai < AR; ++ai) {
    const int a = a0 + ai;
    float pr[8];
    if (a < M) {
      const bool re = a <= cc;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float2 xa = (FULL || j < nv) ? xg[j * M + a] : make_float2(0.f, 0.f);
        // Re(x_a conj x_c) for a <= c, Im(x_c conj x_a) = xa.x*xc.y - xa.y*xc.x for a > c
        pr[j] = fmaf(xa.x, re ? xc[j].x : xc[j].y, xa.y * (re ? xc[j].y : -xc[j].x));
      }
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) pr[j] = 0.f;
    }
    uint4 hv, lv;
    split8(pr, hv, lv);
    const uint32_t off = obase + (uint32_t)((arow0 + ai) * 128);
    *reinterpret_cast<uint4*>(Ah + off) = hv;
    *reinterpret_cast<uint4*>(Al + off) = lv;
  }
}

// barrier 1 over the formation warps only (the MMA warp does not take part), with the OR of
// a per-thread flag: the formation warps take a timeout decision together at it
__device__ __forceinline__ bool formation_sync_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(v ? 1u : 0u), "n"(kScmThreads)
      : "memory");
  return r != 0;
}

// EXACT: M == MAXM (a compile-time channel count in the address arithmetic).
// Warps 0-3 form the operands and own the TMEM lanes (accumulator rows); warp 4 issues the
// input copies (IN stages ahead) and the MMAs.  They meet only at mbarriers:
//   xbar[i]: the inputs of the stage in input buffer i landed (TMA transaction count);
//   rbar[i]: the operands of the stage in operand buffer i are formed (128 arrivals), which
//            also frees that stage's input buffer;
//   mbar[i]: the MMAs of the stage in operand buffer i completed (tcgen05.commit).
// A wait that runs out ends the waiting warp's loop; the CTA then meets at one barrier, and
// one thread waits (with the full bound) for the last MMAs the MMA warp committed before the
// TMEM is freed.
template <int MAXM, bool EXACT>
__global__ void __launch_bounds__(kScmThreads + 32, 4) k_scm_tc(Prob p, int S, int span, int lam_tma,
                                                                const __grid_constant__ CUtensorMap tm_lam) {
  using C = ScmCfg<MAXM>;
  constexpr int KC = C::KC;
  extern __shared__ __align__(1024) unsigned char ssm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ __align__(8) uint64_t xbar[ScmCfg<MAXM>::IN];
  __shared__ __align__(8) uint64_t rbar[2];
  __shared__ __align__(8) uint64_t never_bar;  // nothing arrives here (test limit only)
  __shared__ int s_to, s_mma_last;             // a wait ran out; last stage with committed MMAs
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int F = p.F, T = p.T, N = p.N;
  const int M = EXACT ? MAXM : p.M;
  const int GS = 8 * M + 2;  // complex values per staged 8-frame group
  const int f0 = blockIdx.x * C::FG;
  const int s = blockIdx.y;
  const int tbeg = s * span, tend = min(T, tbeg + span);
  const int nst = tend > tbeg ? (tend - tbeg + KC - 1) / KC : 0;
  const int nbins = min(C::FG, F - f0);
  const int LB = C::lam_bytes(N);
  const bool lam_s = LB > 0;
  // X rows (bin f, frames from t) start at byte 8*M*(f*T + t) and lambda rows at byte
  // 4*((n*F + f)*T + t): with t a multiple of 8 both are 16-byte aligned for every row iff
  // T*M is even and T is a multiple of 4, and so are the copy lengths nf*M*8 and nt*4.
  const bool use_tma = ((T * M) & 1) == 0 && (T & 3) == 0;
  const int IN_BYTES = C::X_BYTES + LB;
  auto xbuf = [&](int c) { return reinterpret_cast<float2*>(ssm + 2 * C::OPS + (c % C::IN) * IN_BYTES); };
  auto lbuf = [&](int c) { return reinterpret_cast<float*>(ssm + 2 * C::OPS + (c % C::IN) * IN_BYTES + C::X_BYTES); };
  float* gs = reinterpret_cast<float*>(ssm + 2 * C::OPS + C::IN * IN_BYTES);  // g~ [FG][N][MAXM]
  constexpr int MMA_WARP = kScmThreads / 32;

  if (warp == 0) { tmem_alloc(&tbase, C::TCOLS); tmem_relinquish(); }
  if (tid == 0) {
    mbar_init(&mbar[0], 1); mbar_init(&mbar[1], 1);
    for (int i = 0; i < C::IN; ++i) mbar_init(&xbar[i], 1);
    mbar_init(&rbar[0], kScmThreads); mbar_init(&rbar[1], kScmThreads);
    mbar_init(&never_bar, 1);
    s_to = 0;
    s_mma_last = -1;
  }
  for (int e = tid; e < C::FG * N * MAXM; e += kScmThreads + 32) {
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

  if (warp == MMA_WARP) {
    // ------------------------------ input copies and MMAs ------------------------------
    auto issue_in = [&](int c) {  // TMA of stage c's X rows (per 8-frame group) and lambda rows
      const int t0 = tbeg + c * KC, nt = min(KC, tend - t0);
      const int ng = (nt + 7) >> 3;
      fence_async_smem();  // the formation warps' generic reads of this buffer came first
      uint64_t* xb = &xbar[c % C::IN];
      // lambda: one tiled copy of the (KC frames x FG bins x N sources) box through the tensor
      // map (zero fill past T and F), else one copy per (bin, source) row
      const uint32_t lam_tx = !lam_s ? 0u : lam_tma ? (uint32_t)LB : (uint32_t)(nt * 4 * N * nbins);
      if (lane == 0) {
        mbar_expect_tx(xb, (uint32_t)(nt * M * 8) * (uint32_t)nbins + lam_tx);
        if (lam_s && lam_tma) tma_tile_3d(lbuf(c), &tm_lam, t0, f0, 0, xb);
      }
      __syncwarp();
      for (int e = lane; e < nbins * ng; e += 32) {
        const int g = e / ng, k = e % ng, nf = min(8, nt - 8 * k);
        tma_bulk_g2s(xbuf(c) + (g * C::NFG + k) * GS, p.X + ((size_t)(f0 + g) * T + t0 + 8 * k) * M,
                     (uint32_t)(nf * M * 8), xb);
      }
      if (lam_s && !lam_tma)
        for (int e = lane; e < nbins * N; e += 32) {
          const int g = e / N, n = e % N;
          tma_bulk_g2s(lbuf(c) + (n * C::FG + g) * KC, p.lam + ((size_t)n * F + f0 + g) * T + t0, (uint32_t)(nt * 4), xb);
        }
    };
    int issued = -1;  // last input stage whose copies were issued
    if (use_tma) {
      for (int c = 0; c < min(C::IN, nst); ++c) issue_in(c);
      issued = min(C::IN, nst) - 1;
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
      // then the copies of stage c + IN into stage c's (consumed) input buffer: issuing the
      // MMAs first keeps them off the copies' issue time
      if (use_tma && c + C::IN < nst) { issue_in(c + C::IN); issued = c + C::IN; }
    }
    if (lane == 0) s_mma_last = mma_last;
    if (!ok) {
      if (lane == 0) { atomicOr(p.status, ST_TIMEOUT); s_to = 1; }
      // copies still in flight land before the CTA releases its shared memory (bounded)
      for (int c = max(0, issued - C::IN + 1); c <= issued; ++c)
        mbar_wait(&xbar[c % C::IN], (uint32_t)((c / C::IN) & 1), kMaxTries);
    }
  } else {
    // ------------------------------ operand formation ------------------------------
    // register accumulators: this thread's TMEM lane = A row r -> (bin g, product q)
    const int r = tid;
    const int rg = r / (8 * MAXM), rrem = r % (8 * MAXM);
    const int ra = rrem >> 3, rlow = rrem & 7;
    const int rgl = rlow / MAXM, rc = rlow % MAXM;
    const int rbin = rg * C::GL + rgl;
    const int rq = ra * MAXM + rc;
    const int colw = ((32 * warp) / (8 * MAXM)) * C::GL * MAXM;  // first accumulator column this warp reads
    const int coff = rbin * MAXM - colw;                         // this lane's bin within those columns
    float vacc[MAXM];
#pragma unroll
    for (int m = 0; m < MAXM; ++m) vacc[m] = 0.f;
    auto flush = [&](int blk) {  // add the accumulator of block blk (its MMAs are complete)
      const uint32_t ta = tacc + ((uint32_t)(32 * warp) << 16) + (uint32_t)((blk & 1) * C::NC + colw);
      float v[C::NCW];
      if (C::NCW == 16) tmem_ld16(ta, v);
      else tmem_ld8(ta, v);
#pragma unroll
      for (int j = 0; j < C::NCW; ++j) {
        const int m = j - coff;
#pragma unroll
        for (int mm = 0; mm < MAXM; ++mm)
          if (m == mm) vacc[mm] += v[j];
      }
    };

    // this thread's product item: (bin g, channel c, frame group, a-range)
    constexpr int AR = MAXM / C::AP;
    const int a_low = tid & 7, a_fgrp = (tid >> 3) % C::NFG, a_rest = (tid >> 3) / C::NFG;
    const int a_ap = a_rest % C::AP, a_gq = a_rest / C::AP;
    const int a_g = a_gq * C::GL + a_low / MAXM, a_c = a_low % MAXM;
    const bool a_ok = (a_g < nbins) && (a_c < M);
    const uint32_t a_obase = (uint32_t)(a_fgrp * (128 * 16) + a_low * 16);
    // this thread's weight item: (bin g, channel m, frame group); row = g*MAXM + m.  With
    // fewer items than threads every WS-th thread takes one, so that all warps share them.
    constexpr int WS = kScmThreads / C::NB_ITEMS;
    const int w_e = tid / WS;
    const int w_low = w_e & 7, w_fgrp = (w_e >> 3) % C::NFG, w_gq = (w_e >> 3) / C::NFG;
    const int w_row = w_gq * 8 + w_low, w_g = w_row / MAXM, w_m = w_row % MAXM;
    const bool w_item = (tid % WS) == 0;
    const bool w_ok = w_item && (w_g < nbins) && (w_m < M);
    const uint32_t w_off = (uint32_t)(w_fgrp * (C::NC * 16) + (w_row >> 3) * 128 + (w_row & 7) * 16);

    int c = 0;
    for (; c < nst; ++c) {
      const int t0 = tbeg + c * KC, nt = min(KC, tend - t0);
      unsigned char* st = ssm + (c & 1) * C::OPS;
      unsigned char* Ah = st;
      unsigned char* Al = st + C::A_BYTES;
      unsigned char* Bh = st + 2 * C::A_BYTES;
      unsigned char* Bl = Bh + C::B_BYTES;
      // the MMAs of stage c-2 read this operand buffer (and those before it are done too)
      // decisions are warp-uniform at least: flush() reads TMEM with a warp-collective load
      const bool to = c >= 2 && !__all_sync(0xffffffffu, mbar_wait(&mbar[c & 1], (uint32_t)(((c - 2) >> 1) & 1), lim));
      tc_fence_after();
      // the block that ended with stage c-2 goes into the registers
      if (!to && c >= 2 && (c - 2) % C::SPB == C::SPB - 1) flush((c - 2) / C::SPB);
      float2* xs = xbuf(c);
      float* ls = lbuf(c);
      if (use_tma) {
        // no barrier among the formation warps on this path: each may leave on its own
        if (to || !__all_sync(0xffffffffu, mbar_wait(&xbar[c % C::IN], (uint32_t)((c / C::IN) & 1), lim))) {
          ok = false;
          break;
        }
      } else {
        for (int e = tid; e < nbins * nt * M; e += kScmThreads) {
          const int g = e / (nt * M), j = e - g * (nt * M), t = j / M;
          xs[(g * C::NFG + (t >> 3)) * GS + (t & 7) * M + (j - t * M)] = p.X[((size_t)(f0 + g) * T + t0) * M + j];
        }
        if (lam_s)
          for (int e = tid; e < nbins * N * nt; e += kScmThreads) {
            const int gn = e / nt, t = e - gn * nt, g = gn / N, n = gn % N;
            ls[(n * C::FG + g) * KC + t] = p.lam[((size_t)n * F + f0 + g) * T + t0 + t];
          }
        if (formation_sync_or(to)) { ok = false; break; }  // leave together
      }

      // ---- B operand: 1/y~ of 8 frames per (bin, channel); y~ written to the state ----
      if (w_item) {
        const int nv = min(8, nt - 8 * w_fgrp);  // valid frames of this group (may be <= 0)
        float y[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) y[j] = 0.f;
        if (w_ok && nv > 0) {
          const size_t pt0 = (size_t)(f0 + w_g) * T + t0 + 8 * w_fgrp;
          for (int n = 0; n < N; ++n) {
            const float gv = gs[(w_g * N + n) * MAXM + w_m];
            float l[8];
            if (lam_s) {
              const float4 l0 = *reinterpret_cast<const float4*>(ls + (n * C::FG + w_g) * KC + 8 * w_fgrp);
              const float4 l1 = *reinterpret_cast<const float4*>(ls + (n * C::FG + w_g) * KC + 8 * w_fgrp + 4);
              l[0] = l0.x; l[1] = l0.y; l[2] = l0.z; l[3] = l0.w; l[4] = l1.x; l[5] = l1.y; l[6] = l1.z; l[7] = l1.w;
            } else {
#pragma unroll
              for (int j = 0; j < 8; ++j) l[j] = (j < nv) ? __ldg(p.lam + (size_t)n * F * T + pt0 + j) : 0.f;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) y[j] = fmaf(l[j], gv, y[j]);
          }
          float* yp = p.yt + pt0 * M + w_m;
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (j < nv) yp[j * M] = y[j];
        }
        float w[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) w[j] = (w_ok && j < nv) ? __fdividef(1.f, y[j]) : 0.f;
        uint4 hv, lv;
        split8(w, hv, lv);
        *reinterpret_cast<uint4*>(Bh + w_off) = hv;
        *reinterpret_cast<uint4*>(Bl + w_off) = lv;
      }

      // ---- A operand: products of 8 frames per (bin, c, frame group, a range) ----
      {
        const int nv = min(8, nt - 8 * a_fgrp);
        const float2* xg = xs + (a_g * C::NFG + a_fgrp) * GS;
        if (a_ok && nv == 8)
          form_products<MAXM, AR, true>(xg, M, 8, a_c, a_ap * AR, Ah, Al, a_obase, a_gq * MAXM + a_ap * AR);
        else
          form_products<MAXM, AR, false>(xg, M, a_ok ? nv : 0, a_c, a_ap * AR, Ah, Al, a_obase, a_gq * MAXM + a_ap * AR);
      }
      // operands visible to the tensor core, then hand the stage to the MMA warp
      fence_async_smem();
      tc_fence_before();
      mbar_arrive(&rbar[c & 1]);
    }
    const int ndone = c;  // stages this thread formed
    if (ok && ndone >= 1) {
      // all MMAs: wait for the last stage's commit (completion is in issue order)
      if (!__all_sync(0xffffffffu, mbar_wait(&mbar[(ndone - 1) & 1], (uint32_t)(((ndone - 1) >> 1) & 1), lim)))
        ok = false;
      tc_fence_after();
      if (ok) {
        const int last = (ndone - 1) / C::SPB;
        // block last-1 was flushed in the loop only if the stage after its successor ran
        if (last >= 1 && ndone == last * C::SPB + 1) flush(last - 1);
        flush(last);
      }
    }
    if (!ok) {
      if (lane == 0) { atomicOr(p.status, ST_TIMEOUT); s_to = 1; }
    } else {
      const int f = f0 + rbin;
      if (rbin < nbins && rc < M && ra < M) {
        float* part = p.part + (size_t)s * F * M * C::MM;
#pragma unroll
        for (int m = 0; m < MAXM; ++m)
          if (m < M) part[((size_t)f * M + m) * C::MM + rq] = vacc[m];
      }
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
}

}  // namespace fm
