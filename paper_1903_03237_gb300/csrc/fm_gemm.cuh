// Batched tensor-core GEMM on tcgen05 (BF16 or TF32 operands, FP32 accumulation in TMEM):
//
//   C[s][b][i][j] = sum_{k in split s} A(b, i, k) * B(b, j, k)
//
// A and B are read from global memory (float32) through arbitrary element strides, rounded
// to the MMA operand type and staged by the CTA's threads into shared memory in the
// K-major core-matrix layout (fm_tc.cuh); a transposed source is therefore as cheap as a
// contiguous one.  One CTA computes a 128 x NT tile of C (MMA M = 128, N = NT), looping
// over its split of the K dimension in chunks of 64; two shared-memory stages let the
// threads fill one stage while the tensor core works on the other.  One thread issues the
// MMAs and commits them to an mbarrier per stage; every wait is bounded and reports
// ST_TIMEOUT instead of hanging.
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
};

__host__ __device__ inline int gemm_stage_bytes(int nt, bool tf32) {
  const int es = tf32 ? 4 : 2;
  return (128 + nt) * kGemmKc * es;
}

template <int NT, bool TF32>
__global__ void __launch_bounds__(kGemmThreads) k_gemm_tc(GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char gsm[];
  constexpr int ES = TF32 ? 4 : 2;
  constexpr int KB = kGemmKc * ES;                  // bytes per row per stage
  constexpr int A_BYTES = 128 * KB, B_BYTES = NT * KB;
  constexpr int STAGE = A_BYTES + B_BYTES;
  constexpr uint32_t TCOLS = NT < 32 ? 32 : NT;      // TMEM columns (power of two >= 32)
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = blockIdx.x * 128, j0 = blockIdx.y * NT;
  const int b = blockIdx.z / g.ksplit, s = blockIdx.z % g.ksplit;
  const int kbeg = s * g.kspan, kend = min(g.Kd, kbeg + g.kspan);
  const float* A = g.A + (long long)b * g.sAb;
  const float* B = g.B + (long long)(b % g.bmodB) * g.sBb;

  if (warp == 0) { tmem_alloc(&tbase, TCOLS); tmem_relinquish(); }
  if (tid == 0) { mbar_init(&mbar[0], 1); mbar_init(&mbar[1], 1); }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tacc = tbase;
  constexpr uint32_t idesc = TF32 ? idesc_tf32_f32(128, NT) : idesc_bf16_f32(128, NT);
  constexpr uint32_t kMaxTries = 1u << 20;

  bool ok = true;
  int c = 0;
  for (int k0 = kbeg; k0 < kend; k0 += kGemmKc, ++c) {
    unsigned char* st = gsm + (c & 1) * STAGE;
    if (c >= 2) {  // the MMAs of chunk c-2 read this stage: wait for them
      if (!mbar_wait(&mbar[c & 1], (uint32_t)(((c - 2) >> 1) & 1), kMaxTries)) { ok = false; break; }
    }
    const int kn = min(kGemmKc, kend - k0);
    // stage A (128 x kn) and B (NT x kn): the stride-1 index runs along the lanes
    auto stage = [&](const float* src, long long sr, long long sk, int rows, int r0, int rlim, unsigned char* dst) {
      if (sk == 1) {
        for (int e = tid; e < rows * kGemmKc; e += kGemmThreads) {
          const int r = e / kGemmKc, k = e % kGemmKc;
          float v = 0.f;
          if (r0 + r < rlim && k < kn) v = src[(long long)(r0 + r) * sr + (k0 + k)];
          if (TF32) *reinterpret_cast<float*>(dst + cm_offset(r, k, KB, 4)) = to_tf32(v);
          else *reinterpret_cast<__nv_bfloat16*>(dst + cm_offset(r, k, KB, 2)) = __float2bfloat16_rn(v);
        }
      } else {
        for (int e = tid; e < rows * kGemmKc; e += kGemmThreads) {
          const int k = e / rows, r = e % rows;
          float v = 0.f;
          if (r0 + r < rlim && k < kn) v = src[(long long)(r0 + r) * sr + (long long)(k0 + k) * sk];
          if (TF32) *reinterpret_cast<float*>(dst + cm_offset(r, k, KB, 4)) = to_tf32(v);
          else *reinterpret_cast<__nv_bfloat16*>(dst + cm_offset(r, k, KB, 2)) = __float2bfloat16_rn(v);
        }
      }
    };
    stage(A, g.sAi, g.sAk, 128, i0, g.Mr, st);
    stage(B, g.sBj, g.sBk, NT, j0, g.Nc, st + A_BYTES);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      const uint32_t sa = smem_u32(st), sb = smem_u32(st + A_BYTES);
      constexpr int KSTEP = 32;  // bytes of K per MMA (16 BF16 or 8 TF32 elements)
#pragma unroll
      for (int q = 0; q < KB / KSTEP; ++q) {
        const uint64_t da = umma_desc(sa + q * 2 * 128, 128, (KB / 16) * 128);
        const uint64_t db = umma_desc(sb + q * 2 * 128, 128, (KB / 16) * 128);
        if (TF32) umma_tf32(tacc, da, db, idesc, (c > 0 || q > 0) ? 1u : 0u);
        else umma_f16(tacc, da, db, idesc, (c > 0 || q > 0) ? 1u : 0u);
      }
      umma_commit(&mbar[c & 1]);
    }
  }
  const int nchunks = c;
  // wait for the last one or two chunks
  if (ok && nchunks >= 2 && !mbar_wait(&mbar[(nchunks - 2) & 1], (uint32_t)(((nchunks - 2) >> 1) & 1), kMaxTries)) ok = false;
  if (ok && nchunks >= 1 && !mbar_wait(&mbar[(nchunks - 1) & 1], (uint32_t)(((nchunks - 1) >> 1) & 1), kMaxTries)) ok = false;
  tc_fence_after();
  if (!ok) {
    if (lane == 0) atomicOr(g.status, ST_TIMEOUT);
  } else if (nchunks > 0) {
    // epilogue: warp w holds rows 32w..32w+31 of the tile
    const int i = i0 + 32 * warp + lane;
    float* Cb = g.C + (long long)s * g.sCs + (long long)b * g.sCb;
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
    float* Cb = g.C + (long long)s * g.sCs + (long long)b * g.sCb;
    if (i < g.Mr)
      for (int j = j0; j < min(g.Nc, j0 + NT); ++j) Cb[(long long)i * g.sCi + (long long)j * g.sCj] = 0.f;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tacc, TCOLS);
}

}  // namespace fm
