// Front end of the paper's experiments (Sec. IV-A): the STFT (window of L = 1024 points, so
// F = 513, and a shift of 256 points in the paper; any power of two L from 16 to 4096 and any
// shift here), its inverse by weighted overlap-add, and the initialisation of g~ and Q by
// spectral decomposition of the initial SCMs.  The paper names neither the window nor the
// framing: a periodic Hann window w_j = (1 - cos(2 pi j / L)) / 2, frames starting at sample
// t * hop with zeros past the end, and synthesis with the same window normalised by the
// overlap-added squared window are this library's reading.
//
//   k_stft        one CTA per (frame, channel): the windowed frame in shared memory in
//                 bit-reversed order, an iterative radix-2 FFT (twiddles by sincospif of exact
//                 dyadic arguments), bins 0..L/2 written to X[f][t][m];
//   k_istft       one CTA per (frame, channel, source): the Hermitian spectrum, the inverse
//                 FFT, the real part times the window into a frame buffer;
//   k_ola         one thread per output sample: the frames covering it added in frame order
//                 and divided by the overlap-added squared window (no atomics: deterministic);
//   k_spec_init   one thread per bin: G_1f = (1/T) sum_t x x^H in float64, its
//                 eigendecomposition by cyclic Jacobi rotations, Q_f = U_f^H (rows the
//                 conjugated eigenvectors, largest eigenvalue first), g~_1f the eigenvalues,
//                 g~_nf = 1 (Q_f I Q_f^H = I), then the nu normalisation with w (or lambda)
//                 scaled to match.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "fastmnmf.h"
#include "fm_common.cuh"
#include "fm_launch.h"

namespace {

using namespace fm;

constexpr int kFeThreads = 256;

fmnmf_status fe_err(fmnmf_status s, const char* fmt, ...) {
  char buf[384];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  fm::set_thread_error(buf);
  return s;
}

int ilog2(int L) {
  int l = 0;
  while ((1 << l) < L) ++l;
  return l;
}

__device__ __forceinline__ float hann_w(int j, int L) { return 0.5f - 0.5f * cospif(2.0f * (float)j / (float)L); }

// In-place iterative radix-2 FFT of z[0..L) (input in bit-reversed order, output in natural
// order); sign -1: forward (e^{-2 pi i f j / L}), +1: inverse (unscaled).
__device__ void fft_smem(float2* z, int L, int lg, float sign) {
  for (int s = 1; s <= lg; ++s) {
    const int half = 1 << (s - 1);
    __syncthreads();
    for (int b = threadIdx.x; b < L / 2; b += blockDim.x) {
      const int k = b & (half - 1);
      const int i0 = ((b >> (s - 1)) << s) + k, i1 = i0 + half;
      float sn, cs;
      sincospif(sign * (float)k / (float)half, &sn, &cs);  // exact dyadic argument
      const float2 a = z[i0], c = z[i1];
      const float2 t = make_float2(cs * c.x - sn * c.y, cs * c.y + sn * c.x);
      z[i0] = make_float2(a.x + t.x, a.y + t.y);
      z[i1] = make_float2(a.x - t.x, a.y - t.y);
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kFeThreads) k_stft(const float* __restrict__ x, int M, int S, int L, int lg, int hop,
                                                    int T, float2* __restrict__ X) {
  extern __shared__ float2 zs[];
  const int t = blockIdx.x, m = blockIdx.y;
  for (int j = threadIdx.x; j < L; j += blockDim.x) {
    const int s = t * hop + j;
    const float v = (s < S) ? x[(size_t)m * S + s] * hann_w(j, L) : 0.f;
    zs[__brev((unsigned)j) >> (32 - lg)] = make_float2(v, 0.f);
  }
  fft_smem(zs, L, lg, -1.f);
  const int F = L / 2 + 1;
  for (int f = threadIdx.x; f < F; f += blockDim.x) X[((size_t)f * T + t) * M + m] = zs[f];
}

__global__ void __launch_bounds__(kFeThreads) k_istft(const float2* __restrict__ Y, int F, int T, int M, int L, int lg,
                                                     float* __restrict__ fr) {
  extern __shared__ float2 zs[];
  const int t = blockIdx.x, m = blockIdx.y, b = blockIdx.z;
  const float2* Yb = Y + (size_t)b * F * T * M;
  for (int k = threadIdx.x; k < L; k += blockDim.x) {
    float2 v;
    if (k <= L / 2) {
      v = Yb[((size_t)k * T + t) * M + m];
      if (k == 0 || k == L / 2) v.y = 0.f;  // the real bins (as an inverse real DFT takes them)
    } else {
      const float2 c = Yb[((size_t)(L - k) * T + t) * M + m];
      v = make_float2(c.x, -c.y);
    }
    zs[__brev((unsigned)k) >> (32 - lg)] = v;
  }
  fft_smem(zs, L, lg, 1.f);
  const float inv = 1.f / (float)L;
  float* out = fr + (((size_t)b * M + m) * T + t) * L;
  for (int j = threadIdx.x; j < L; j += blockDim.x) out[j] = zs[j].x * inv * hann_w(j, L);
}

__global__ void __launch_bounds__(kFeThreads) k_ola(const float* __restrict__ fr, int B, int M, int T, int L, int hop,
                                                   int S, float thr, float* __restrict__ y) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)B * M * S) return;
  const int s = (int)(i % S);
  const size_t bm = i / S;
  const float* base = fr + bm * T * L;
  const int t_lo = s < L ? 0 : (s - L) / hop + 1;
  const int t_hi = min(T - 1, s / hop);
  float acc = 0.f, den = 0.f;
  for (int t = t_lo; t <= t_hi; ++t) {
    const int j = s - t * hop;
    const float w = hann_w(j, L);
    acc += base[(size_t)t * L + j];
    den = fmaf(w, w, den);
  }
  y[i] = den > thr ? acc / den : 0.f;
}

// Cyclic Jacobi eigendecomposition of a Hermitian matrix A (M <= kMaxM, row-major in local
// memory) in float64: A <- J^H A J with J[p][p] = J[q][q] = c, J[p][q] = s e, J[q][p] = -s e*
// (e the phase of A[p][q], t = tan of the rotation angle from (A_qq - A_pp) / (2 |A_pq|)),
// which zeroes A[p][q]; V <- V J accumulates the eigenvectors (columns).
__device__ void herm_jacobi(double2 (*A)[kMaxM], double2 (*V)[kMaxM], int M) {
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) V[i][j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int i = 0; i < M; ++i)
      for (int j = 0; j < M; ++j) {
        const double a2 = A[i][j].x * A[i][j].x + A[i][j].y * A[i][j].y;
        if (i == j) dia += a2; else off += a2;
      }
    if (!(off > 1e-30 * dia)) break;
    for (int p = 0; p < M - 1; ++p)
      for (int q = p + 1; q < M; ++q) {
        const double2 apq = A[p][q];
        const double r = sqrt(apq.x * apq.x + apq.y * apq.y);
        if (!(r > 1e-300)) continue;
        const double2 e = make_double2(apq.x / r, apq.y / r);
        const double tau = (A[q][q].x - A[p][p].x) / (2.0 * r);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
        // J entries: jpq = s e, jqp = -s conj(e)
        const double2 jpq = make_double2(sn * e.x, sn * e.y), jqp = make_double2(-sn * e.x, sn * e.y);
        // A <- A J (columns p, q)
        for (int i = 0; i < M; ++i) {
          const double2 aip = A[i][p], aiq = A[i][q];
          A[i][p] = make_double2(c * aip.x + (aiq.x * jqp.x - aiq.y * jqp.y), c * aip.y + (aiq.x * jqp.y + aiq.y * jqp.x));
          A[i][q] = make_double2((aip.x * jpq.x - aip.y * jpq.y) + c * aiq.x, (aip.x * jpq.y + aip.y * jpq.x) + c * aiq.y);
          const double2 vip = V[i][p], viq = V[i][q];
          V[i][p] = make_double2(c * vip.x + (viq.x * jqp.x - viq.y * jqp.y), c * vip.y + (viq.x * jqp.y + viq.y * jqp.x));
          V[i][q] = make_double2((vip.x * jpq.x - vip.y * jpq.y) + c * viq.x, (vip.x * jpq.y + vip.y * jpq.x) + c * viq.y);
        }
        // A <- J^H A (rows p, q): (J^H)[p][q] = conj(jqp), (J^H)[q][p] = conj(jpq)
        for (int j = 0; j < M; ++j) {
          const double2 apj = A[p][j], aqj = A[q][j];
          const double2 hpq = make_double2(jqp.x, -jqp.y), hqp = make_double2(jpq.x, -jpq.y);
          A[p][j] = make_double2(c * apj.x + (hpq.x * aqj.x - hpq.y * aqj.y), c * apj.y + (hpq.x * aqj.y + hpq.y * aqj.x));
          A[q][j] = make_double2((hqp.x * apj.x - hqp.y * apj.y) + c * aqj.x, (hqp.x * apj.y + hqp.y * apj.x) + c * aqj.y);
        }
      }
  }
}

// One thread per bin; lam: the lambda state of the unconstrained model (else null).
__global__ void __launch_bounds__(128) k_spec_init(Prob p, float* __restrict__ lam) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  const int F = p.F, T = p.T, M = p.M, N = p.N, K = p.K;
  if (f >= F) return;
  double2 A[kMaxM][kMaxM], V[kMaxM][kMaxM];
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) A[i][j] = make_double2(0.0, 0.0);
  const float2* xf = p.X + (size_t)f * T * M;
  for (int t = 0; t < T; ++t) {
    double2 xv[kMaxM];
    for (int j = 0; j < M; ++j) {
      const float2 v = xf[(size_t)t * M + j];
      xv[j] = make_double2(v.x, v.y);
    }
    for (int i = 0; i < M; ++i)
      for (int j = 0; j < M; ++j) {  // x_i conj(x_j)
        A[i][j].x += xv[i].x * xv[j].x + xv[i].y * xv[j].y;
        A[i][j].y += xv[i].y * xv[j].x - xv[i].x * xv[j].y;
      }
  }
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) A[i][j] = make_double2(A[i][j].x / T, A[i][j].y / T);
  herm_jacobi(A, V, M);
  // eigenvalues largest first (selection order; ties keep the lower index)
  int ord[kMaxM];
  bool used[kMaxM];
  for (int i = 0; i < M; ++i) used[i] = false;
  for (int r = 0; r < M; ++r) {
    int best = -1;
    for (int i = 0; i < M; ++i)
      if (!used[i] && (best < 0 || A[i][i].x > A[best][best].x)) best = i;
    ord[r] = best;
    used[best] = true;
  }
  // Q_f rows: conjugated eigenvectors (Q = U^H), float-float storage
  for (int r = 0; r < M; ++r)
    for (int j = 0; j < M; ++j) {
      const double2 v = V[j][ord[r]];
      const double re = v.x, im = -v.y;
      const float rh = (float)re, ih = (float)im;
      p.Qx[((size_t)f * M + r) * M + j] = make_float4(rh, (float)(re - rh), ih, (float)(im - ih));
    }
  // g~: eigenvalues for source 1, ones for the others; nu normalisation, w or lambda scaled
  double nu0 = 0.0;
  for (int r = 0; r < M; ++r) nu0 += fmax(A[ord[r]][ord[r]].x, 0.0);
  if (!(nu0 > 0.0) || !isfinite(nu0)) flag(p.status, ST_SINGULAR);
  for (int n = 0; n < N; ++n) {
    const double nu = n == 0 ? nu0 : (double)M;
    for (int r = 0; r < M; ++r)
      p.G[((size_t)n * F + f) * M + r] = (float)(n == 0 ? fmax(A[ord[r]][ord[r]].x, 0.0) / nu : 1.0 / M);
    if (lam) {
      for (int t = 0; t < T; ++t) lam[((size_t)n * F + f) * T + t] = (float)(lam[((size_t)n * F + f) * T + t] * nu);
    } else {
      for (int k = 0; k < K; ++k) p.W[((size_t)n * K + k) * F + f] = (float)(p.W[((size_t)n * K + k) * F + f] * nu);
    }
  }
}

bool dev_ptr(const void* p) {
  cudaPointerAttributes a;
  return cudaPointerGetAttributes(&a, p) == cudaSuccess && (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
}

}  // namespace

namespace fm {
cudaError_t launch_spec_init(const Prob& p, float* lam, cudaStream_t st) {
  k_spec_init<<<(p.F + 127) / 128, 128, 0, st>>>(p, lam);
  return cudaGetLastError();
}
}  // namespace fm

namespace {

fmnmf_status check_frame_args(int L, int hop, int S, const char* who) {
  if (L < 16 || L > 4096 || (L & (L - 1)))
    return fe_err(FMNMF_EINVAL, "%s: L = %d must be a power of two in [16, 4096]", who, L);
  if (hop < 1 || hop > L) return fe_err(FMNMF_EINVAL, "%s: hop = %d must be in [1, L]", who, hop);
  if (S < 1) return fe_err(FMNMF_EINVAL, "%s: S = %d must be >= 1", who, S);
  return FMNMF_OK;
}

int frames_of(int S, int L, int hop) { return S <= L ? 1 : 1 + (int)(((long long)S - L + hop - 1) / hop); }

}  // namespace

extern "C" {

fmnmf_status fmnmf_stft_frames(int S, int L, int hop, int* T) {
  fmnmf_status s = check_frame_args(L, hop, S, "stft_frames");
  if (s != FMNMF_OK) return s;
  if (!T) return fe_err(FMNMF_EINVAL, "stft_frames: T is NULL");
  *T = frames_of(S, L, hop);
  return FMNMF_OK;
}

fmnmf_status fmnmf_stft(const float* x, int M, int S, int L, int hop, void* X, void* stream) {
  fmnmf_status s = check_frame_args(L, hop, S, "stft");
  if (s != FMNMF_OK) return s;
  if (M < 1 || M > 65535) return fe_err(FMNMF_EINVAL, "stft: M = %d must be in [1, 65535]", M);
  if (!x || !X) return fe_err(FMNMF_EINVAL, "stft: NULL pointer");
  if (((uintptr_t)x & 3) || ((uintptr_t)X & 7)) return fe_err(FMNMF_EINVAL, "stft: x must be 4-byte and X 8-byte aligned");
  if (!dev_ptr(x) || !dev_ptr(X)) return fe_err(FMNMF_EINVAL, "stft: x and X must be device pointers");
  const int T = frames_of(S, L, hop);
  if (T > 0x7fffffff / 2) return fe_err(FMNMF_EINVAL, "stft: too many frames");
  const cudaStream_t st = (cudaStream_t)stream;
  k_stft<<<dim3(T, M), kFeThreads, (size_t)L * sizeof(float2), st>>>(x, M, S, L, ilog2(L), hop, T, (float2*)X);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fe_err(FMNMF_ECUDA, "stft launch: %s", cudaGetErrorString(e));
  return FMNMF_OK;
}

fmnmf_status fmnmf_istft(const void* Y, int B, int F, int T, int M, int S, int L, int hop, float* y, void* stream) {
  fmnmf_status s = check_frame_args(L, hop, S, "istft");
  if (s != FMNMF_OK) return s;
  if (F != L / 2 + 1) return fe_err(FMNMF_EINVAL, "istft: F = %d must be L/2 + 1 = %d", F, L / 2 + 1);
  if (B < 1 || B > 65535 || M < 1 || M > 65535 || T < 1)
    return fe_err(FMNMF_EINVAL, "istft: B = %d, M = %d must be in [1, 65535] and T = %d >= 1", B, M, T);
  if ((long long)(T - 1) * hop + L < S)
    return fe_err(FMNMF_EINVAL, "istft: %d frames of hop %d cover fewer than S = %d samples", T, hop, S);
  if (!Y || !y) return fe_err(FMNMF_EINVAL, "istft: NULL pointer");
  if (((uintptr_t)Y & 7) || ((uintptr_t)y & 3)) return fe_err(FMNMF_EINVAL, "istft: Y must be 8-byte and y 4-byte aligned");
  if (!dev_ptr(Y) || !dev_ptr(y)) return fe_err(FMNMF_EINVAL, "istft: Y and y must be device pointers");
  // threshold of the squared-window sum: 1e-10 of its largest value over the frames' span
  const long long n_out = (long long)(T - 1) * hop + L;
  double dmax = 0.0;
  const long long lim = std::min<long long>(n_out, (long long)L + 2LL * L);  // the sum is hop-periodic inside
  for (long long sidx = 0; sidx < lim; ++sidx) {
    double d = 0.0;
    const long long t_lo = sidx < L ? 0 : (sidx - L) / hop + 1, t_hi = std::min<long long>(T - 1, sidx / hop);
    for (long long t = t_lo; t <= t_hi; ++t) {
      const double w = 0.5 - 0.5 * std::cos(2.0 * M_PI * (double)(sidx - t * hop) / L);
      d += w * w;
    }
    dmax = std::max(dmax, d);
  }
  const float thr = (float)(1e-10 * dmax);
  const cudaStream_t st = (cudaStream_t)stream;
  const size_t fr_bytes = (size_t)B * M * T * L * sizeof(float);
  float* fr = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&fr, fr_bytes, st);
  if (e != cudaSuccess) return fe_err(FMNMF_ENOMEM, "istft: frame buffer (%zu bytes): %s", fr_bytes, cudaGetErrorString(e));
  k_istft<<<dim3(T, M, B), kFeThreads, (size_t)L * sizeof(float2), st>>>((const float2*)Y, F, T, M, L, ilog2(L), fr);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    const size_t n = (size_t)B * M * S;
    k_ola<<<(unsigned)((n + kFeThreads - 1) / kFeThreads), kFeThreads, 0, st>>>(fr, B, M, T, L, hop, S, thr, y);
    e = cudaGetLastError();
  }
  cudaFreeAsync(fr, st);
  if (e != cudaSuccess) return fe_err(FMNMF_ECUDA, "istft launch: %s", cudaGetErrorString(e));
  return FMNMF_OK;
}

}  // extern "C"
