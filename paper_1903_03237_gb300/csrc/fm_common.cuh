// Device-side definitions shared by the FastMNMF kernels (sm_103a).
//
// Notation follows Sekiguchi et al. 2019 (arXiv 1903.03237): F bins, T frames, M channels,
// N sources, K NMF bases; W[n][k][f], H[n][k][t], g~ = G[n][f][m], Q[f][m][j] with row m of
// Q_f = q_fm^H (Eq. 16), x~ = xt[f][t][m] = |Q_f x_ft|^2, y~ = yt[f][t][m] = sum_n lambda g~.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fm {

constexpr int kThreads = 256;   // every tiled kernel runs 256 threads (8 warps)
constexpr int kOT = 8;          // "own" elements (bins or frames) per CTA tile; one warp per element in the IP
constexpr int kMaxM = 8;        // channels supported

enum : unsigned { ST_NONFINITE = 1u, ST_SINGULAR = 2u, ST_TIMEOUT = 4u };

// Everything a kernel needs to know about one mixture's device state.
struct Prob {
  int F, T, M, N, K;
  const float2* X;     // [F][T][M] complex64 mixture
  float* W;            // [N][K][F]
  float* H;            // [N][K][T]
  float* G;            // [N][F][M]
  float4* Qx;          // [F][M][M] diagonalisers, float-float (re.hi, re.lo, im.hi, im.lo)
  float4* Qix;         // [F][M][M] their inverses, float-float (carried by the IP update)
  float2* Qf;          // [F][M][M] float32 copy of Q used by the sweeps
  float2* Qinv;        // [F][M][M] float32 copy of Q^-1 (Wiener filter)
  float* xt;           // [F][T][M] projected powers x~
  float* yt;           // [F][T][M] model powers y~
  double* logdet;      // [F] log|det Q_f|^2 (carried by the IP update)
  float* phi;          // [F] tr(Q_f Q_f^H)/M of the last IP update (1 if none)
  double* ll;          // [1] log-likelihood of the current state
  unsigned* status;    // [1] sticky ST_* bits
  float* part;         // split-sum partials (sized by the host for the largest user)
  double* llpart;      // [ll_blocks] per-CTA log-likelihood partials
  unsigned* counters;  // arrival counters of the split reductions (zero between launches)
  const float* lam;    // [N][F][T] lambda formed by the tensor-core GEMM (mixed form), or null
  float* nu_out;       // [N][F] nu_nf of the normalisation written by k_bin, or null
  unsigned wait_limit; // 0: the normal bound of the tensor-core kernels' waits; else a test
                       // limit for their consumer waits, with one wait on an mbarrier nothing
                       // arrives at (makes the timeout path run; drains keep the full bound)
};

// Tiling of a launch over (own tile) x (inner split): own = the index the update writes
// (f for W, g~, V; t for H), inner = the index summed over (t for W, g~, V; f for H).
struct Geom {
  int n_own_tiles;  // ceil(own extent / kOT)
  int S;            // inner splits (gridDim.y)
  int span;         // inner elements per split, multiple of 4
  int IC;           // inner elements staged per sub-chunk, multiple of 4
  int ICP;          // padded smem row (IC + 4 floats: keeps 16-byte rows on distinct banks)
};

// ---- small complex helpers ---------------------------------------------------------
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  double d = 1.0 / cabs2(b);
  return make_double2((a.x * b.x + a.y * b.y) * d, (a.y * b.x - a.x * b.y) * d);
}

__device__ __forceinline__ void flag(unsigned* status, unsigned bits) { atomicOr(status, bits); }

// Split-reduction arrival: every CTA of a group calls this after writing its partials;
// returns true in exactly one CTA (the last to arrive), which then reads all partials.
// Partials must be read with __ldcg (L2) by the last CTA.
__device__ __forceinline__ bool arrive_last(unsigned* counter, unsigned expected) {
  __shared__ unsigned s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(counter, 1u);
    s_last = (prev == expected - 1u);
    if (s_last) *counter = 0u;  // ready for the next launch
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0u;
}

}  // namespace fm
