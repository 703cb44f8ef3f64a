// Batched tensor-core GEMM on tcgen05 (BF16 or TF32 operands, FP32 accumulation in TMEM):
//
//   C[s][b][i][j] = sum_{k in split s} A(b, i, k) * B(b, j, k)
//
// A and B are read from global memory (float32) through arbitrary element strides, rounded
// to the MMA operand type and staged by the CTA's threads into shared memory in the
// K-major core-matrix layout (k-groups outermost); a transposed source is therefore as
// cheap as a contiguous one.  BF16 operands are split: v = hi + lo with hi = bf16(v) and
// lo = bf16(v - hi), and each product is taken as hi*hi + hi*lo + lo*hi (three MMAs into
// the same accumulator; the lo*lo term is below 2^-16 of the product), which carries about
// 16 significant bits of each operand; the two tiles take the bytes one TF32 tile takes.  The epilogue goes through shared memory so that every store
// instruction writes whole row segments of C.  One CTA computes a 128 x NT tile of C
// (MMA M = 128, N = NT), looping over its split of the K dimension in chunks of 64; two shared-memory stages let the
// threads fill one stage while the tensor core works on the other.  One thread issues the
// MMAs and commits them to an mbarrier per stage; every wait is bounded and reports
// ST_TIMEOUT instead of hanging.  The CTA takes a timeout decision together (a barrier with
// an OR of the threads' results), then waits, with the full bound, for the MMAs it committed
// before it frees its TMEM.
#pragma once
#include <cuda_bf16.h>

#include "fm_common.cuh"
#include "fm_tc.cuh"

namespace fm {

constexpr int kGemmKc = 64;        // K elements per stage
constexpr int kGemmThreads = 128;  // 4 warps: one per 32 TMEM lanes

struct GemmArgs {
  const float* A; long long sAb, sAi, sAk;  // element strides of A(b, i, k)
  const float* B; long long sBb, sBj, sBk;  // element strides of B(b, j, k)
  int bmodB;                                 // B batch index = b % bmodB
  float* C; long long sCs, sCb, sCi, sCj;   // output (split s, batch b, row i, column j)
  int Mr, Nc, Kd, batch, ksplit, kspan;      // kspan = K elements per split (multiple of kGemmKc)
  unsigned* status;
  unsigned wait_limit;                       // test limit of the consumer waits (0: normal), see Prob
};

// Bytes of one pipeline stage: the A and B tiles (TF32), or their hi and lo BF16 tiles.
__host__ __device__ inline int gemm_stage_bytes(int nt, bool tf32) {
  (void)tf32;
  return (128 + nt) * kGemmKc * 4;
}

// Stages a rows x kGemmKc tile of src(r0 + r, k0 + k) (zero outside [rlim) x [kn)) as BF16 or
// TF32 into the K-major core-matrix layout with the 16-byte k-groups outermost: core row
// (r, kg) at byte (kg * rows + r) * 16.  A thread builds whole 16-byte rows (8 BF16 or 4
// TF32 values); consecutive threads take consecutive r, so the stores fill all banks.  The
// loads are float4 when the tile rows are contiguous in k and 16-byte aligned (vec), else
// scalar (consecutive threads then read consecutive r, which is the stride-1 index when
// the rows are not contiguous in k).  A thread issues the loads of up to 8 rows before
// converting and storing any of them, so that many loads are in flight.
template <bool TF32, int ROWS>
struct StageShape {
  static constexpr int EPG = TF32 ? 4 : 8;              // values per 16-byte core row
  static constexpr int KG = kGemmKc / EPG;
  static constexpr int ITEMS = ROWS * KG / kGemmThreads;  // 16-byte rows per thread
  static constexpr int BATCH = ITEMS < 8 ? ITEMS : 8;     // loads issued together (in flight at once)
  static_assert(ITEMS * kGemmThreads == ROWS * KG, "whole rows per thread");
};

// Loads the values of a thread's 16-byte rows i0 .. i0 + BATCH - 1 of the tile (see
// gemm_stage_tile) into v; nothing is converted or stored yet.
template <bool TF32, int ROWS>
__device__ __forceinline__ void gemm_tile_load(const float* __restrict__ src, long long sr, long long sk, int r0,
                                               int rlim, int k0, int kn, bool vec, int i0,
                                               float (&v)[StageShape<TF32, ROWS>::BATCH][StageShape<TF32, ROWS>::EPG]) {
  using Sh = StageShape<TF32, ROWS>;
  constexpr int EPG = Sh::EPG;
#pragma unroll
  for (int u = 0; u < Sh::BATCH; ++u) {
    const int e = (i0 + u) * kGemmThreads + threadIdx.x;
    const int r = e % ROWS, kk = (e / ROWS) * EPG;
    const bool rok = r0 + r < rlim;
    const float* p = src + (long long)(r0 + r) * sr + (long long)(k0 + kk) * sk;
    if (rok && vec && kk + EPG <= kn) {
#pragma unroll
      for (int q = 0; q < EPG / 4; ++q) {
        const float4 x = __ldg(reinterpret_cast<const float4*>(p) + q);
        v[u][4 * q] = x.x; v[u][4 * q + 1] = x.y; v[u][4 * q + 2] = x.z; v[u][4 * q + 3] = x.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < EPG; ++j) v[u][j] = (rok && kk + j < kn) ? __ldg(p + (long long)j * sk) : 0.f;
    }
  }
}

// Rounds the loaded rows to TF32, or splits them into BF16 hi and lo parts (lo tile at
// dst + lo_off), and stores them as core rows.
__device__ __forceinline__ uint32_t bf16x2_bits(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}
template <bool TF32, int ROWS>
__device__ __forceinline__ void gemm_tile_store(int i0, const float (&v)[StageShape<TF32, ROWS>::BATCH][StageShape<TF32, ROWS>::EPG],
                                                unsigned char* dst, int lo_off) {
  using Sh = StageShape<TF32, ROWS>;
  constexpr int EPG = Sh::EPG;
#pragma unroll
  for (int u = 0; u < Sh::BATCH; ++u) {
    const int e = (i0 + u) * kGemmThreads + threadIdx.x;
    const int r = e % ROWS, kg = e / ROWS;
    if (TF32) {
      const uint4 o = make_uint4(__float_as_uint(to_tf32(v[u][0])), __float_as_uint(to_tf32(v[u][1])),
                                 __float_as_uint(to_tf32(v[u][2])), __float_as_uint(to_tf32(v[u][3])));
      *reinterpret_cast<uint4*>(dst + (kg * ROWS + r) * 16) = o;
    } else {
      float hi[8], lo[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        hi[q] = __bfloat162float(__float2bfloat16_rn(v[u][q % EPG]));
        lo[q] = v[u][q % EPG] - hi[q];  // exact in float32
      }
      const uint4 oh = make_uint4(bf16x2_bits(hi[0], hi[1]), bf16x2_bits(hi[2], hi[3]), bf16x2_bits(hi[4], hi[5]),
                                  bf16x2_bits(hi[6], hi[7]));
      const uint4 ol = make_uint4(bf16x2_bits(lo[0], lo[1]), bf16x2_bits(lo[2], lo[3]), bf16x2_bits(lo[4], lo[5]),
                                  bf16x2_bits(lo[6], lo[7]));
      *reinterpret_cast<uint4*>(dst + (kg * ROWS + r) * 16) = oh;
      *reinterpret_cast<uint4*>(dst + lo_off + (kg * ROWS + r) * 16) = ol;
    }
  }
}

// Stages a rows x kGemmKc tile of src(r0 + r, k0 + k) (zero outside [rlim) x [kn)) as BF16 or
// TF32 into the K-major core-matrix layout with the 16-byte k-groups outermost: core row
// (r, kg) at byte (kg * rows + r) * 16.  A thread builds whole 16-byte rows (8 BF16 or 4
// TF32 values); consecutive threads take consecutive r, so the stores fill all banks.  The
// loads are float4 when the tile rows are contiguous in k and 16-byte aligned (vec), else
// scalar (consecutive threads then read consecutive r, which is the stride-1 index when
// the rows are not contiguous in k).  A thread issues the loads of up to 8 rows before
// converting and storing any of them, so that many loads are in flight.
template <bool TF32, int ROWS>
__device__ __forceinline__ void gemm_stage_tile(const float* __restrict__ src, long long sr, long long sk, int r0,
                                                int rlim, int k0, int kn, bool vec, unsigned char* dst, int lo_off) {
  using Sh = StageShape<TF32, ROWS>;
#pragma unroll 1
  for (int i0 = 0; i0 < Sh::ITEMS; i0 += Sh::BATCH) {
    float v[Sh::BATCH][Sh::EPG];
    gemm_tile_load<TF32, ROWS>(src, sr, sk, r0, rlim, k0, kn, vec, i0, v);
    gemm_tile_store<TF32, ROWS>(i0, v, dst, lo_off);
  }
}

template <int NT, bool TF32>
__global__ void __launch_bounds__(kGemmThreads) k_gemm_tc(GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char gsm[];
  constexpr int ES = TF32 ? 4 : 2;
  constexpr int KB = kGemmKc * ES;                  // bytes per row per stage
  constexpr int A_BYTES = 128 * KB, B_BYTES = NT * KB;
  constexpr int LO = A_BYTES + B_BYTES;              // BF16: the lo tiles follow the hi tiles
  constexpr int STAGE = TF32 ? A_BYTES + B_BYTES : 2 * (A_BYTES + B_BYTES);
  constexpr uint32_t TCOLS = NT < 32 ? 32 : NT;      // TMEM columns (power of two >= 32)
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ __align__(8) uint64_t never_bar;  // nothing arrives here (test limit only)
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = blockIdx.x * 128, j0 = blockIdx.y * NT;
  const int b = blockIdx.z / g.ksplit, s = blockIdx.z % g.ksplit;
  const int kbeg = s * g.kspan, kend = min(g.Kd, kbeg + g.kspan);
  const float* A = g.A + (long long)b * g.sAb;
  const float* B = g.B + (long long)(b % g.bmodB) * g.sBb;
  // float4 operand loads: rows contiguous in k, row starts 16-byte aligned (k0 is a
  // multiple of kGemmKc and the k-groups of 4)
  const bool vecA = g.sAk == 1 && (g.sAi & 3) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
  const bool vecB = g.sBk == 1 && (g.sBj & 3) == 0 && (reinterpret_cast<uintptr_t>(B) & 15) == 0;

  if (warp == 0) { tmem_alloc(&tbase, TCOLS); tmem_relinquish(); }
  if (tid == 0) { mbar_init(&mbar[0], 1); mbar_init(&mbar[1], 1); mbar_init(&never_bar, 1); }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tacc = tbase;
  constexpr uint32_t idesc = TF32 ? idesc_tf32_f32(128, NT) : idesc_bf16_f32(128, NT);
  constexpr uint32_t kMaxTries = 1u << 22;
  const uint32_t lim = g.wait_limit ? g.wait_limit : kMaxTries;  // consumer waits

  bool ok = true;
  int c = 0;
  using SA = StageShape<TF32, 128>;
  using SB = StageShape<TF32, NT>;
  // Small tiles (BF16, NT <= 32: both operands in one batch each): the loads of A and B are
  // in flight together; with NT = 32 a chunk's loads are also issued while the previous
  // chunk's barrier and MMAs run (held across them, the registers would cut the occupancy
  // of the narrower tile and of wider ones).
  constexpr bool kCombine = SA::ITEMS == SA::BATCH && SB::ITEMS == SB::BATCH && SA::ITEMS + SB::ITEMS <= 10;
  constexpr bool kPipe = kCombine && NT == 32;
  float va[SA::BATCH][SA::EPG], vb[SB::BATCH][SB::EPG];
  if constexpr (kPipe) {
    if (kbeg < kend) {
      const int kn0 = min(kGemmKc, kend - kbeg);
      gemm_tile_load<TF32, 128>(A, g.sAi, g.sAk, i0, g.Mr, kbeg, kn0, vecA, 0, va);
      gemm_tile_load<TF32, NT>(B, g.sBj, g.sBk, j0, g.Nc, kbeg, kn0, vecB, 0, vb);
    }
  }
  for (int k0 = kbeg; k0 < kend; k0 += kGemmKc, ++c) {
    unsigned char* st = gsm + (c & 1) * STAGE;
    // the MMAs of chunk c-2 read this stage: wait for them (after a timeout the stores below
    // may overwrite operands still being read: results are then flagged, memory stays in bounds)
    const bool to = c >= 2 && !mbar_wait(&mbar[c & 1], (uint32_t)(((c - 2) >> 1) & 1), lim);
    const int kn = min(kGemmKc, kend - k0);
    if constexpr (kPipe) {
      gemm_tile_store<TF32, 128>(0, va, st, LO);
      gemm_tile_store<TF32, NT>(0, vb, st + A_BYTES, LO);
      const int k1 = k0 + kGemmKc;
      if (k1 < kend) {
        const int kn1 = min(kGemmKc, kend - k1);
        gemm_tile_load<TF32, 128>(A, g.sAi, g.sAk, i0, g.Mr, k1, kn1, vecA, 0, va);
        gemm_tile_load<TF32, NT>(B, g.sBj, g.sBk, j0, g.Nc, k1, kn1, vecB, 0, vb);
      }
    } else if constexpr (kCombine) {
      gemm_tile_load<TF32, 128>(A, g.sAi, g.sAk, i0, g.Mr, k0, kn, vecA, 0, va);
      gemm_tile_load<TF32, NT>(B, g.sBj, g.sBk, j0, g.Nc, k0, kn, vecB, 0, vb);
      gemm_tile_store<TF32, 128>(0, va, st, LO);
      gemm_tile_store<TF32, NT>(0, vb, st + A_BYTES, LO);
    } else {
      gemm_stage_tile<TF32, 128>(A, g.sAi, g.sAk, i0, g.Mr, k0, kn, vecA, st, LO);
      gemm_stage_tile<TF32, NT>(B, g.sBj, g.sBk, j0, g.Nc, k0, kn, vecB, st + A_BYTES, LO);
    }
    fence_async_smem();
    tc_fence_before();
    if (__syncthreads_or(to ? 1 : 0)) { ok = false; break; }  // the whole CTA leaves together
    tc_fence_after();
    if (tid == 0) {
      const uint32_t sa = smem_u32(st), sb = smem_u32(st + A_BYTES);
      constexpr uint32_t ALBO = 128 * 16, BLBO = NT * 16;
#pragma unroll
      for (int q = 0; q < KB / 32; ++q) {  // 32 bytes of K per MMA (16 BF16 or 8 TF32)
        const uint64_t da = umma_desc(sa + q * 2 * ALBO, ALBO, 128);
        const uint64_t db = umma_desc(sb + q * 2 * BLBO, BLBO, 128);
        if (TF32) {
          umma_tf32(tacc, da, db, idesc, (c > 0 || q > 0) ? 1u : 0u);
        } else {
          const uint64_t dal = umma_desc(sa + LO + q * 2 * ALBO, ALBO, 128);
          const uint64_t dbl = umma_desc(sb + LO + q * 2 * BLBO, BLBO, 128);
          umma_f16(tacc, da, db, idesc, (c > 0 || q > 0) ? 1u : 0u);  // hi * hi
          umma_f16(tacc, da, dbl, idesc, 1u);                          // hi * lo
          umma_f16(tacc, dal, db, idesc, 1u);                          // lo * hi
        }
      }
      umma_commit(&mbar[c & 1]);
    }
  }
  const int nchunks = c;  // chunks whose MMAs were committed (the same in every thread)
  // wait for the last one or two chunks
  bool to = !ok;
  if (!to && g.wait_limit) to = !mbar_wait(&never_bar, 0u, lim);  // test limit: runs out
  if (!to && nchunks >= 2) to = !mbar_wait(&mbar[(nchunks - 2) & 1], (uint32_t)(((nchunks - 2) >> 1) & 1), lim);
  if (!to && nchunks >= 1) to = !mbar_wait(&mbar[(nchunks - 1) & 1], (uint32_t)(((nchunks - 1) >> 1) & 1), lim);
  if (__syncthreads_or(to ? 1 : 0)) {
    ok = false;
    // drain: every committed MMA lands before TMEM is freed (completion is in issue order)
    if (nchunks >= 1) mbar_wait(&mbar[(nchunks - 1) & 1], (uint32_t)(((nchunks - 1) >> 1) & 1), kMaxTries);
  }
  tc_fence_after();
  float* Cb = g.C + (long long)s * g.sCs + (long long)b * g.sCb;
  if (!ok) {
    if (lane == 0) atomicOr(g.status, ST_TIMEOUT);
  } else if (nchunks > 0 && g.sCj == 1) {
    // epilogue through shared memory (free: every MMA has completed): warp w holds rows
    // 32w..32w+31 of the tile; it writes CW columns of its 32 rows at a time, each store
    // instruction covering whole row segments (each warp uses its own scratch rows)
    constexpr int CW = NT < 32 ? NT : 32;
    constexpr int RPI = 32 / CW;  // rows per store instruction
    float* scr = reinterpret_cast<float*>(gsm) + warp * (32 * 33);
    const int lc = lane % CW, lr = lane / CW;
#pragma unroll 1
    for (int cc = 0; cc < NT; cc += CW) {
      float v[CW];
      tmem_ld16(tacc + ((uint32_t)(32 * warp) << 16) + (uint32_t)cc, v);
      if (CW == 32) tmem_ld16(tacc + ((uint32_t)(32 * warp) << 16) + (uint32_t)(cc + 16), v + (CW == 32 ? 16 : 0));
#pragma unroll
      for (int q = 0; q < CW; ++q) scr[lane * 33 + q] = v[q];
      __syncwarp();
      const int j = j0 + cc + lc;
#pragma unroll 4
      for (int rr = lr; rr < 32; rr += RPI) {
        const int i = i0 + 32 * warp + rr;
        if (i < g.Mr && j < g.Nc) Cb[(long long)i * g.sCi + j] = scr[rr * 33 + lc];
      }
      __syncwarp();
    }
  } else if (nchunks > 0) {
    // epilogue: warp w holds rows 32w..32w+31 of the tile
    const int i = i0 + 32 * warp + lane;
#pragma unroll
    for (int cc = 0; cc < NT; cc += 16) {
      float v[16];
      tmem_ld16(tacc + ((uint32_t)(32 * warp) << 16) + (uint32_t)cc, v);
      if (i < g.Mr) {
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int j = j0 + cc + jj;
          if (j < g.Nc) Cb[(long long)i * g.sCi + (long long)j * g.sCj] = v[jj];
        }
      }
    }
  } else {
    // empty split: zero output
    const int i = i0 + 32 * warp + lane;
    if (i < g.Mr)
      for (int j = j0; j < min(g.Nc, j0 + NT); ++j) Cb[(long long)i * g.sCi + (long long)j * g.sCj] = 0.f;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tacc, TCOLS);
}

}  // namespace fm
