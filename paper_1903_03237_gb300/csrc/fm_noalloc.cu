// fmnmf_loglik_noalloc: the log-likelihood of Eq. 17 for a state held in the caller's own
// device buffers, without allocating any memory.
//
// Some callers cannot call cudaMalloc: a real-time audio thread must not block, and
// cudaMalloc may wait for the device for an unbounded time; an application whose device
// memory is owned entirely by its own pool allocator does not let a library take memory
// behind its back.  This entry point serves them.  It is a variant of the x~ /
// log-likelihood kernel of the context path (k_xt_ll): that kernel's per-CTA partial sums
// and arrival counter, and the per-bin log|det Q_f|^2 it reads, live here in one
// file-scope static device array instead of a context's arena.
//
// The array (kScratchBytes, 1 MiB) exists on every device that loads the library, until
// the process exits.  Every call shares it and it keeps the last call's contents, so the
// counter is cleared at the start of each call; calls that overlap on the GPU race for
// it and must be ordered by the caller (same stream, or events).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <string>

#include "fastmnmf.h"
#include "fm_kernels.cuh"
#include "fm_launch.h"

namespace {

using namespace fm;

constexpr size_t kScratchBytes = size_t(1) << 20;
constexpr int kNaMaxF = 16384;                       // bins: log-det slots
constexpr int kNaPtsPerBlock = kThreads * kPtsPerThread;
constexpr size_t kNaLogdetBytes = (size_t)kNaMaxF * sizeof(double);
constexpr size_t kNaCounterOffset = kNaLogdetBytes;  // one unsigned, padded to 256 bytes
constexpr size_t kNaPartOffset = kNaCounterOffset + 256;
constexpr int kNaMaxBlocks = (int)((kScratchBytes - kNaPartOffset) / sizeof(double));
constexpr int kNaCacheSlots = 64;

static __device__ __align__(256) unsigned char g_na_scratch[kScratchBytes];

// The array's device address differs between driver contexts (the module is loaded again
// after cudaDeviceReset, and each context that shares a device has its own copy), so the
// cache is keyed on the current context's unique ID (cuCtxGetId: never reused within the
// process, unlike a context handle), not on the device number.
struct NaSlot {
  unsigned long long id;
  void* ptr;
};
std::mutex g_na_mu;
NaSlot g_na_cache[kNaCacheSlots] = {};
int g_na_next = 0;

// Errors are reported through fmnmf_last_error(NULL), like every context-less failure.
fmnmf_status na_err(fmnmf_status s, const char* fmt, ...) {
  char buf[384];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  fm::set_thread_error(buf);
  return s;
}

// cuCtxGetCurrent and cuCtxGetId through the runtime's driver entry points (no link-time
// libcuda dependency).
struct CtxFns {
  PFN_cuCtxGetCurrent_v4000 current = nullptr;
  PFN_cuCtxGetId_v12000 id = nullptr;
};
const CtxFns& ctx_fns() {
  static CtxFns fns;
  static std::once_flag once;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &ptr, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fns.current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(ptr);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fns.id = reinterpret_cast<PFN_cuCtxGetId_v12000>(ptr);
  });
  return fns;
}

// ID of the current context (0 when the thread has none yet).
bool current_ctx_id(unsigned long long* id) {
  const CtxFns& f = ctx_fns();
  CUcontext cur = nullptr;
  if (!f.current || !f.id || f.current(&cur) != CUDA_SUCCESS) return false;
  *id = 0;
  return !cur || f.id(cur, id) == CUDA_SUCCESS;
}

// Device address of the scratch array in the current context: looked up with
// cudaGetSymbolAddress the first time a context calls (with its device current) and cached
// per context.  A thread with no current context yet gets the device's primary context
// from that lookup (the runtime binds it), and the context is read again afterwards.
fmnmf_status na_scratch(void** out) {
  unsigned long long id = 0;
  if (!current_ctx_id(&id)) return na_err(FMNMF_ECUDA, "cuCtxGetCurrent / cuCtxGetId failed");
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (id)
    for (const NaSlot& s : g_na_cache)
      if (s.ptr && s.id == id) { *out = s.ptr; return FMNMF_OK; }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
  if (e != cudaSuccess || !p) return na_err(FMNMF_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
  if (!current_ctx_id(&id) || !id) return na_err(FMNMF_ECUDA, "no current CUDA context");
  g_na_cache[g_na_next] = NaSlot{id, p};  // the oldest slot makes room
  g_na_next = (g_na_next + 1) % kNaCacheSlots;
  *out = p;
  return FMNMF_OK;
}

// log|det Q_f|^2 per bin (float64 LU), one warp per bin, into the scratch log-det slots.
template <int MAXM>
__global__ void __launch_bounds__(kThreads) k_na_logdet(const float2* __restrict__ Q, int F, int M,
                                                        double* __restrict__ logdet) {
  __shared__ double2 A_s[kThreads / 32][MAXM * MAXM];
  __shared__ double2 fac_s[kThreads / 32][MAXM];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int f = blockIdx.x * (kThreads / 32) + warp;
  if (f >= F) return;
  double2* A = A_s[warp];
  for (int e = lane; e < M * M; e += 32) {
    const float2 v = Q[(size_t)f * M * M + e];
    A[(e / M) * MAXM + e % M] = make_double2(v.x, v.y);
  }
  __syncwarp();
  const double ld = warp_logdet2(M, MAXM, A, fac_s[warp]);
  if (lane == 0) logdet[f] = ld;
}

// Per point: lambda_ftn = sum_k w h (Eq. 9), y~ (below Eq. 17), x~ = |Q_f x_ft|^2, and the
// term -x~/y~ - log y~; per-CTA sums in the scratch; the last CTA adds T sum_f log-det and
// the constant -F T M log(pi) and writes *ll.
template <int MAXM>
__global__ void __launch_bounds__(kThreads) k_na_loglik(const float2* __restrict__ X, const float* __restrict__ W,
                                                        const float* __restrict__ H, const float* __restrict__ G,
                                                        const float2* __restrict__ Q, int F, int T, int M, int N, int K,
                                                        const double* __restrict__ logdet, double* part,
                                                        unsigned* counter, double* ll) {
  const int tid = threadIdx.x;
  const size_t npts = (size_t)F * T;
  float acc = 0.f;
  for (int r = 0; r < kPtsPerThread; ++r) {
    const size_t pt = (size_t)blockIdx.x * kNaPtsPerBlock + (size_t)r * kThreads + tid;
    if (pt >= npts) break;
    const int f = (int)(pt / T), t = (int)(pt % T);
    float y[MAXM];
#pragma unroll
    for (int m = 0; m < MAXM; ++m) y[m] = 0.f;
    for (int n = 0; n < N; ++n) {
      float lam = 0.f;
      for (int k = 0; k < K; ++k) lam = fmaf(W[((size_t)n * K + k) * F + f], H[((size_t)n * K + k) * T + t], lam);
#pragma unroll
      for (int m = 0; m < MAXM; ++m)
        if (m < M) y[m] = fmaf(lam, G[((size_t)n * F + f) * M + m], y[m]);
    }
    float2 x[MAXM];
#pragma unroll
    for (int j = 0; j < MAXM; ++j) x[j] = (j < M) ? X[pt * M + j] : make_float2(0.f, 0.f);
    const float2* q = Q + (size_t)f * M * M;
#pragma unroll
    for (int m = 0; m < MAXM; ++m) {
      if (m < M) {
        float re = 0.f, im = 0.f;
#pragma unroll
        for (int j = 0; j < MAXM; ++j)
          if (j < M) {
            const float2 a = q[m * M + j];
            re = fmaf(a.x, x[j].x, fmaf(-a.y, x[j].y, re));
            im = fmaf(a.x, x[j].y, fmaf(a.y, x[j].x, im));
          }
        const float xv = re * re + im * im;
        acc += -xv / y[m] - logf(y[m]);
      }
    }
  }
  __shared__ double red[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((tid & 31) == 0) red[tid >> 5] = (double)acc;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    part[blockIdx.x] = s;
  }
  if (!arrive_last(counter, gridDim.x)) return;
  double s = 0.0, ld = 0.0;
  for (int b = tid; b < (int)gridDim.x; b += kThreads) s += __ldcg(part + b);
  for (int f = tid; f < F; f += kThreads) ld += __ldcg(logdet + f);
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    ld += __shfl_xor_sync(0xffffffffu, ld, o);
  }
  __shared__ double red2[2][kThreads / 32];
  __syncthreads();
  if ((tid & 31) == 0) { red2[0][tid >> 5] = s; red2[1][tid >> 5] = ld; }
  __syncthreads();
  if (tid == 0) {
    double S = 0.0, LD = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) { S += red2[0][w]; LD += red2[1][w]; }
    *ll = S + (double)T * LD - (double)F * T * M * 1.1447298858494002;  // log(pi)
  }
}

template <int MAXM>
cudaError_t na_launch(const float2* X, const float* W, const float* H, const float* G, const float2* Q, int F,
                      int T, int M, int N, int K, double* ll, char* scratch, int nblk, cudaStream_t st) {
  double* logdet = reinterpret_cast<double*>(scratch);
  unsigned* counter = reinterpret_cast<unsigned*>(scratch + kNaCounterOffset);
  double* part = reinterpret_cast<double*>(scratch + kNaPartOffset);
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st);  // clear what must start at zero
  if (e != cudaSuccess) return e;
  constexpr int kBinsPerBlock = kThreads / 32;  // one warp per bin
  k_na_logdet<MAXM><<<(F + kBinsPerBlock - 1) / kBinsPerBlock, kThreads, 0, st>>>(Q, F, M, logdet);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_na_loglik<MAXM><<<nblk, kThreads, 0, st>>>(X, W, H, G, Q, F, T, M, N, K, logdet, part, counter, ll);
  return cudaGetLastError();
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

}  // namespace

extern "C" fmnmf_status fmnmf_loglik_noalloc(const void* X, const float* W, const float* H, const float* G,
                                             const void* Q, int F, int T, int M, int N, int K, double* ll,
                                             void* stream) {
  if (!X || !W || !H || !G || !Q || !ll) return na_err(FMNMF_EINVAL, "loglik_noalloc: NULL pointer");
  if (F < 1 || T < 1 || M < 1 || M > kMaxM || N < 1 || K < 1)
    return na_err(FMNMF_EINVAL, "loglik_noalloc: bad shape F=%d T=%d M=%d N=%d K=%d", F, T, M, N, K);
  if (F > kNaMaxF)
    return na_err(FMNMF_EINVAL, "loglik_noalloc: F=%d exceeds the scratch limit of %d bins", F, kNaMaxF);
  const size_t npts = (size_t)F * T;
  const size_t nblk = (npts + kNaPtsPerBlock - 1) / kNaPtsPerBlock;
  if (nblk > (size_t)kNaMaxBlocks)
    return na_err(FMNMF_EINVAL, "loglik_noalloc: F*T=%zu exceeds the scratch limit of %zu TF bins", npts,
                  (size_t)kNaMaxBlocks * kNaPtsPerBlock);
  if (!aligned(X, 8) || !aligned(Q, 8) || !aligned(W, 4) || !aligned(H, 4) || !aligned(G, 4) || !aligned(ll, 8))
    return na_err(FMNMF_EINVAL, "loglik_noalloc: misaligned pointer");
  void* scratch = nullptr;
  fmnmf_status s = na_scratch(&scratch);
  if (s != FMNMF_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const float2* Xc = (const float2*)X;
  const float2* Qc = (const float2*)Q;
  char* sc = (char*)scratch;
  cudaError_t e;
  if (M <= 2) e = na_launch<2>(Xc, W, H, G, Qc, F, T, M, N, K, ll, sc, (int)nblk, st);
  else if (M <= 4) e = na_launch<4>(Xc, W, H, G, Qc, F, T, M, N, K, ll, sc, (int)nblk, st);
  else e = na_launch<8>(Xc, W, H, G, Qc, F, T, M, N, K, ll, sc, (int)nblk, st);
  if (e != cudaSuccess) return na_err(FMNMF_ECUDA, "loglik_noalloc launch: %s", cudaGetErrorString(e));
  return FMNMF_OK;
}
