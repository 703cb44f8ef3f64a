// Mixed-precision form of the FastMNMF iteration: the dense contractions run on the
// tensor cores (tcgen05, BF16 or TF32 operands, FP32 accumulation), the rest on the CUDA
// cores in FP32, the IP in float-float.
//
//   lambda_n = W_n^T H_n                     (Eq. 9)      k_gemm_tc  [F x T] per source
//   P, R per TF bin from x~ and y~           (Eqs. 23-24) k_pr for the H update; for the W
//                                                         update the kernel that forms x~
//                                                         (k_ip or k_xt_ll) writes them
//   num/den W_n = [P_n; R_n] H_n^T           (Eq. 23)     k_gemm_tc  sum over t, split-K
//   num/den H_n = [P_n; R_n]^T W_n^T         (Eq. 24)     k_gemm_tc  sum over f, split-K
//   W, H <- W, H * sqrt(num/den)                          k_apply (sums the splits in order)
// The g~ update (Eq. 21, k_g_tc) and V_fm (Eq. 18, k_scm_tc) run on the tensor cores from
// the materialised lambda; the IP, x~, log-likelihood and normalisation kernels are those
// of the plain form.
#include <cuda_runtime.h>

#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>
#include <type_traits>

#include "fm_g_tc.cuh"
#include "fm_gemm.cuh"
#include "fm_kernels.cuh"
#include "fm_launch.h"
#include "fm_scm_tc.cuh"

namespace fm {

// P_n = sum_m g~_nfm x~/y~^2 and R_n = sum_m g~_nfm / y~ per TF bin, into PR[2][N][F][T].
// y~ is read (mode 0, the W update: y~ of the current state is kept in p.yt) or formed from
// the materialised lambda (mode 1, the H update).
template <int MAXM>
__global__ void __launch_bounds__(kThreads) k_pr(Prob p, float* __restrict__ PR, int mode) {
  const int F = p.F, T = p.T, M = p.M, N = p.N;
  const unsigned npts = (unsigned)F * (unsigned)T;
  const unsigned pt = blockIdx.x * (unsigned)kThreads + threadIdx.x;
  if (pt >= npts) return;
  const int f = (int)(pt / (unsigned)T);
  float y[MAXM], x[MAXM];
  if (M == MAXM && MAXM % 4 == 0) {  // whole points as float4
#pragma unroll
    for (int q = 0; q < MAXM / 4; ++q) {
      const float4 v = *reinterpret_cast<const float4*>(p.xt + (size_t)pt * MAXM + 4 * q);
      x[4 * q] = v.x; x[4 * q + 1] = v.y; x[4 * q + 2] = v.z; x[4 * q + 3] = v.w;
      const float4 w = mode == 0 ? *reinterpret_cast<const float4*>(p.yt + (size_t)pt * MAXM + 4 * q)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
      y[4 * q] = w.x; y[4 * q + 1] = w.y; y[4 * q + 2] = w.z; y[4 * q + 3] = w.w;
    }
  } else {
#pragma unroll
    for (int m = 0; m < MAXM; ++m) {
      x[m] = (m < M) ? p.xt[(size_t)pt * M + m] : 0.f;
      y[m] = (mode == 0 && m < M) ? p.yt[(size_t)pt * M + m] : 0.f;
    }
  }
  if (mode == 1) {
    for (int n = 0; n < N; ++n) {
      const float l = p.lam[(size_t)n * npts + pt];
      const float* g = p.G + ((size_t)n * F + f) * M;
#pragma unroll
      for (int m = 0; m < MAXM; ++m)
        if (m < M) y[m] = fmaf(l, g[m], y[m]);
    }
  }
  pr_point<MAXM>(x, y, M, N, p.G + (size_t)f * M, (size_t)F * M, PR, npts, pt);
}

// fac[n][k][o] *= sqrt(num/den) with num = sum_s C[s][n][o][k], den = sum_s C[s][N+n][o][k].
// Threads run along the split buffer's layout (k fastest), so the split loads coalesce.
__global__ void __launch_bounds__(kThreads) k_apply(float* __restrict__ fac, const float* __restrict__ C, int S,
                                                    int N, int K, int own, unsigned* status) {
  const size_t total = (size_t)N * K * own;
  const size_t e = (size_t)blockIdx.x * kThreads + threadIdx.x;
  if (e >= total) return;
  const int k = (int)(e % K);
  const size_t no = e / K;
  const int o = (int)(no % own), n = (int)(no / own);
  const size_t split = (size_t)2 * N * own * K;
  // the splits summed in order; their loads issued eight at a time
  float num = 0.f, den = 0.f;
  const float* cn = C + e;
  const float* cd = C + (size_t)N * own * K + e;
  for (int s0 = 0; s0 < S; s0 += 8) {
    float a[8], b[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      a[u] = (s0 + u < S) ? __ldg(cn + (size_t)(s0 + u) * split) : 0.f;
      b[u] = (s0 + u < S) ? __ldg(cd + (size_t)(s0 + u) * split) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) { num += a[u]; den += b[u]; }
  }
  float* fp = fac + ((size_t)n * K + k) * own + o;
  const float v = *fp * sqrtf(num / den);
  if (!isfinite(v)) atomicOr(status, ST_NONFINITE);
  *fp = v;
}

template <int NT, bool TF32>
static cudaError_t gemm_launch(const GemmArgs& g, dim3 grid, cudaStream_t st) {
  // two pipeline stages when a split has more than one K chunk, else one (more CTAs per SM)
  const size_t smem = (g.kspan > kGemmKc ? 2 : 1) * (size_t)gemm_stage_bytes(NT, TF32);
  k_gemm_tc<NT, TF32><<<grid, kGemmThreads, smem, st>>>(g);
  return cudaGetLastError();
}

template <int NT, bool TF32>
static cudaError_t gemm_configure() {
  return cudaFuncSetAttribute(k_gemm_tc<NT, TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              2 * gemm_stage_bytes(NT, TF32));
}

cudaError_t launch_gemm(const GemmArgs& g, bool tf32, int nt, dim3 grid, cudaStream_t st) {
  if (tf32) {
    switch (nt) {
      case 16: return gemm_launch<16, true>(g, grid, st);
      case 32: return gemm_launch<32, true>(g, grid, st);
      case 64: return gemm_launch<64, true>(g, grid, st);
      default: return gemm_launch<128, true>(g, grid, st);
    }
  }
  switch (nt) {
    case 16: return gemm_launch<16, false>(g, grid, st);
    case 32: return gemm_launch<32, false>(g, grid, st);
    case 64: return gemm_launch<64, false>(g, grid, st);
    default: return gemm_launch<128, false>(g, grid, st);
  }
}

template <int MAXM>
static cudaError_t scm_launch(const Prob& p, int S, int span, const CUtensorMap* tl, cudaStream_t st) {
  using C = ScmCfg<MAXM>;
  const dim3 grid((p.F + C::FG - 1) / C::FG, S);
  CUtensorMap zero;
  std::memset(&zero, 0, sizeof zero);
  const int tma = tl != nullptr;
  if (p.M == MAXM) k_scm_tc<MAXM, true><<<grid, kScmThreads + 32, C::smem(p.N), st>>>(p, S, span, tma, tma ? *tl : zero);
  else k_scm_tc<MAXM, false><<<grid, kScmThreads + 32, C::smem(p.N), st>>>(p, S, span, tma, tma ? *tl : zero);
  return cudaGetLastError();
}
// The kernel's shared memory grows with N (lambda rows and g~ staged per bin): raise the
// function's limit to what this N needs (never lower it: contexts share the function).
template <int MAXM>
static cudaError_t scm_configure(int N) {
  static std::mutex mu;
  static int configured = 0;
  const int need = ScmCfg<MAXM>::smem(N);
  std::lock_guard<std::mutex> lk(mu);
  if (need <= configured) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_scm_tc<MAXM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_scm_tc<MAXM, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
  if (e == cudaSuccess) configured = need;
  return e;
}
template <int MAXM>
static int scm_occ(int N) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_scm_tc<MAXM, true>, kScmThreads + 32, ScmCfg<MAXM>::smem(N)) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

cudaError_t configure_gemm() {
  cudaError_t e;
  if ((e = gemm_configure<16, true>()) != cudaSuccess) return e;
  if ((e = gemm_configure<32, true>()) != cudaSuccess) return e;
  if ((e = gemm_configure<64, true>()) != cudaSuccess) return e;
  if ((e = gemm_configure<128, true>()) != cudaSuccess) return e;
  if ((e = gemm_configure<16, false>()) != cudaSuccess) return e;
  if ((e = gemm_configure<32, false>()) != cudaSuccess) return e;
  if ((e = gemm_configure<64, false>()) != cudaSuccess) return e;
  return gemm_configure<128, false>();
}

cudaError_t launch_scm_tc(int maxm, const Prob& p, int S, int span, const CUtensorMap* tl, cudaStream_t st) {
  if (maxm == 2) return scm_launch<2>(p, S, span, tl, st);
  if (maxm == 4) return scm_launch<4>(p, S, span, tl, st);
  return scm_launch<8>(p, S, span, tl, st);
}

int scm_bins_per_cta(int maxm) { return 128 / (maxm * maxm); }
int scm_frames_per_stage(int maxm) { return maxm == 2 ? ScmCfg<2>::KC : maxm == 4 ? ScmCfg<4>::KC : ScmCfg<8>::KC; }
int scm_smem(int maxm, int N) {
  return maxm == 2 ? ScmCfg<2>::smem(N) : maxm == 4 ? ScmCfg<4>::smem(N) : ScmCfg<8>::smem(N);
}
cudaError_t scm_prepare(int maxm, int N) {
  return maxm == 2 ? scm_configure<2>(N) : maxm == 4 ? scm_configure<4>(N) : scm_configure<8>(N);
}
int scm_occupancy(int maxm, int N) { return maxm == 2 ? scm_occ<2>(N) : maxm == 4 ? scm_occ<4>(N) : scm_occ<8>(N); }

// ---- g~ update on the tensor cores ----
template <int MAXM, int NP>
static cudaError_t gtc_launch(const Prob& p, int S, int span, unsigned ctr, const CUtensorMap* tx,
                              const CUtensorMap* tl, cudaStream_t st) {
  using C = GtcCfg<MAXM, NP>;
  const dim3 grid((p.F + C::FG - 1) / C::FG, S);
  CUtensorMap zero;
  std::memset(&zero, 0, sizeof zero);
  const bool tma = tx != nullptr && tl != nullptr;
  k_g_tc<MAXM, NP><<<grid, kGtcThreads + 32, C::smem(p.N), st>>>(p, S, span, ctr, tma ? 1 : 0, tma ? *tx : zero,
                                                                tma ? *tl : zero);
  return cudaGetLastError();
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  });
  return fn;
}

// lambda [N][F][T] as a 3-D tensor (frames, bins, sources) with a (kc, fg, N) box.
static bool lam_tensor_map(const Prob& p, int kc, int fg, CUtensorMap* tl) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || p.T % 4 != 0 || p.lam == nullptr || p.N > 256) return false;
  const cuuint64_t dl[3] = {(cuuint64_t)p.T, (cuuint64_t)p.F, (cuuint64_t)p.N};
  const cuuint64_t sl[2] = {(cuuint64_t)p.T * 4, (cuuint64_t)p.F * p.T * 4};
  const cuuint32_t bl[3] = {(cuuint32_t)kc, (cuuint32_t)fg, (cuuint32_t)p.N};
  const cuuint32_t el[3] = {1, 1, 1};
  return enc(tl, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)p.lam, dl, sl, bl, el, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

bool scm_tensor_map(int maxm, const Prob& p, CUtensorMap* tl) {
  const int fg = 128 / (maxm * maxm), kc = scm_frames_per_stage(maxm);
  // only when the kernel stages lambda (its stage fits the shared-memory cap)
  if ((maxm == 2 ? ScmCfg<2>::lam_bytes(p.N) : maxm == 4 ? ScmCfg<4>::lam_bytes(p.N) : ScmCfg<8>::lam_bytes(p.N)) == 0)
    return false;
  return lam_tensor_map(p, kc, fg, tl);
}

bool gtc_tensor_maps(int maxm, const Prob& p, CUtensorMap* tx, CUtensorMap* tl) {
  // rows of x~ (T*M floats per bin) and lambda (T floats per source and bin) must start on
  // 16-byte boundaries: T a multiple of 4
  if (p.T % 4 != 0 || p.lam == nullptr || p.N > 256) return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const int FG = 64 / maxm, KC = kGtcKc;
  const cuuint64_t dx[2] = {(cuuint64_t)p.T * p.M, (cuuint64_t)p.F};
  const cuuint64_t sx[1] = {(cuuint64_t)p.T * p.M * 4};
  const cuuint32_t bx[2] = {(cuuint32_t)(KC * p.M), (cuuint32_t)FG};
  const cuuint32_t ex[2] = {1, 1};
  if (enc(tx, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)p.xt, dx, sx, bx, ex, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  return lam_tensor_map(p, KC, FG, tl);
}
template <int MAXM, int NP>
static cudaError_t gtc_configure(int N) {
  static std::mutex mu;
  static int configured = 0;
  const int need = GtcCfg<MAXM, NP>::smem(N);
  std::lock_guard<std::mutex> lk(mu);
  if (need <= configured) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_g_tc<MAXM, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
  if (e == cudaSuccess) configured = need;
  return e;
}
template <int MAXM, int NP>
static int gtc_occ(int N) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_g_tc<MAXM, NP>, kGtcThreads + 32, GtcCfg<MAXM, NP>::smem(N)) !=
      cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}
// The source padding of the kernel for (MAXM, N): a power of two >= N and >= MAXM / 2 (a
// warp reads whole 16-column groups), at most 8; 0 when N is too large for it.
int gtc_np(int maxm, int N) {
  int np = 2;
  while (np < N) np *= 2;
  np = std::max(np, maxm / 2);
  return np <= 8 ? np : 0;
}
template <typename Fn>
static auto gtc_dispatch(int maxm, int np, Fn&& fn) {
  switch (maxm * 16 + np) {
    case 8 * 16 + 4: return fn(std::integral_constant<int, 8>(), std::integral_constant<int, 4>());
    case 8 * 16 + 8: return fn(std::integral_constant<int, 8>(), std::integral_constant<int, 8>());
    case 4 * 16 + 2: return fn(std::integral_constant<int, 4>(), std::integral_constant<int, 2>());
    case 4 * 16 + 4: return fn(std::integral_constant<int, 4>(), std::integral_constant<int, 4>());
    case 4 * 16 + 8: return fn(std::integral_constant<int, 4>(), std::integral_constant<int, 8>());
    case 2 * 16 + 2: return fn(std::integral_constant<int, 2>(), std::integral_constant<int, 2>());
    case 2 * 16 + 4: return fn(std::integral_constant<int, 2>(), std::integral_constant<int, 4>());
    default: return fn(std::integral_constant<int, 2>(), std::integral_constant<int, 8>());
  }
}
cudaError_t launch_g_tc(int maxm, int np, const Prob& p, int S, int span, unsigned ctr, const CUtensorMap* tx,
                        const CUtensorMap* tl, cudaStream_t st) {
  return gtc_dispatch(maxm, np, [&](auto mx, auto n) {
    return gtc_launch<decltype(mx)::value, decltype(n)::value>(p, S, span, ctr, tx, tl, st);
  });
}
cudaError_t gtc_prepare(int maxm, int np, int N) {
  return gtc_dispatch(maxm, np, [&](auto mx, auto n) { return gtc_configure<decltype(mx)::value, decltype(n)::value>(N); });
}
int gtc_occupancy(int maxm, int np, int N) {
  return gtc_dispatch(maxm, np, [&](auto mx, auto n) { return gtc_occ<decltype(mx)::value, decltype(n)::value>(N); });
}
int gtc_smem(int maxm, int np, int N) {
  return gtc_dispatch(maxm, np, [&](auto mx, auto n) { return GtcCfg<decltype(mx)::value, decltype(n)::value>::smem(N); });
}
int gtc_bins_per_cta(int maxm) { return 64 / maxm; }
int gtc_frames_per_stage() { return kGtcKc; }

cudaError_t launch_pr(int maxm, const Prob& p, float* PR, int mode, cudaStream_t st) {
  const unsigned npts = (unsigned)p.F * (unsigned)p.T;
  const dim3 grid((npts + kThreads - 1) / kThreads);
  switch (maxm) {
    case 2: k_pr<2><<<grid, kThreads, 0, st>>>(p, PR, mode); break;
    case 4: k_pr<4><<<grid, kThreads, 0, st>>>(p, PR, mode); break;
    default: k_pr<8><<<grid, kThreads, 0, st>>>(p, PR, mode); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_apply(float* fac, const float* C, int S, int N, int K, int own, unsigned* status,
                         cudaStream_t st) {
  const size_t total = (size_t)N * K * own;
  k_apply<<<(unsigned)((total + kThreads - 1) / kThreads), kThreads, 0, st>>>(fac, C, S, N, K, own, status);
  return cudaGetLastError();
}

}  // namespace fm
