// Host-side launch interface of the FastMNMF kernels (one translation unit per channel
// bucket MAXM in {2, 4, 8}; fm_api.cu dispatches on the bucket).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include "fm_common.cuh"

namespace fm {

enum KernelKind {
  KK_W = 0,      // W update (Eq. 23)
  KK_H = 1,      // H update (Eq. 24)
  KK_G = 2,      // g~ update (Eq. 21) + nu normalisation
  KK_Y = 3,      // y~ refresh, V_fm (Eq. 18), IP (Eqs. 19-20) + phi normalisation
  KK_XT = 4,     // x~, log-likelihood (Eq. 17) (long mixtures), mu normalisation
  KK_PREP = 5,   // per-bin float64 preparation (log-det, Q^-1)
  KK_SEP = 6,    // Wiener filter (Eq. 3)
  KK_IP = 7,     // IP solve (Eqs. 19-20) + per-bin normalisation (+ x~ and log-likelihood terms)
  KK_GL = 8,     // mixed form: lambda = W^T H on the tensor cores
  KK_GW = 9,     // mixed form: W numerator / denominator GEMM
  KK_GH = 10,    // mixed form: H numerator / denominator GEMM
  KK_PR = 11,    // mixed form: P, R per TF bin
  KK_APPLY = 12, // mixed form: multiplicative update from the split GEMM sums
  KK_BIN = 13,   // fused schedule: per-bin g~ / V_fm + IP / normalisation / x~ / LL / next W update
  KK_HGEMM = 14, // fused schedule: H update (split GEMM over bins, last-CTA update)
  KK_COUNT = 15
};

struct LaunchArgs {
  Prob p;
  Geom g;
  dim3 grid;
  size_t smem = 0;
  cudaStream_t st = nullptr;
  int flags = 0;          // k_tile / k_ip flags
  int S = 0;              // k_ip: number of V_fm splits
  unsigned ctr = 0;       // first arrival counter of this launch
  int n_pt_blocks = 0;    // k_xt_ll
  int xt_mode = 0;        // k_ip: also x~ and the log-likelihood of its bin
  int apply_phi = 0;      // k_xt_ll
  int do_mu = 0;          // k_xt_ll
  int ll_bins = 0;        // k_xt_ll: a last block adds up the IP kernel's per-bin log-likelihood terms
  float* pr = nullptr;    // k_ip, k_xt_ll: also form P, R of the next W update here
  int ll_tail = 1;        // k_ip: the last CTA adds up the log-likelihood (0: a later kernel does)
  float2* out = nullptr;  // k_separate
  float* lam = nullptr;   // k_bin: lambda [N][F][T]
};

cudaError_t launch_m2(KernelKind k, const LaunchArgs& a);
cudaError_t launch_m4(KernelKind k, const LaunchArgs& a);
cudaError_t launch_m8(KernelKind k, const LaunchArgs& a);
// Resident CTAs per SM of a kernel class at a dynamic shared-memory size.
int occupancy_m2(KernelKind k, size_t smem);
int occupancy_m4(KernelKind k, size_t smem);
int occupancy_m8(KernelKind k, size_t smem);
// Resident CTAs per SM of the fused-schedule kernels.
int occupancy_fused_m2(KernelKind k, size_t smem);
int occupancy_fused_m4(KernelKind k, size_t smem);
int occupancy_fused_m8(KernelKind k, size_t smem);
// Raises the dynamic shared-memory limit of every kernel of the bucket to `bytes`.
cudaError_t configure_m2(int bytes);
cudaError_t configure_m4(int bytes);
cudaError_t configure_m8(int bytes);

// Mixed-precision form (fm_mixed.cu).
struct GemmArgs;
cudaError_t launch_gemm(const GemmArgs& g, bool tf32, int nt, dim3 grid, cudaStream_t st);
cudaError_t configure_gemm();
cudaError_t launch_pr(int maxm, const Prob& p, float* PR, int mode, cudaStream_t st);
// Spectral initialisation of g~ and Q (front end): writes G, Qx and scales W (or lambda).
cudaError_t launch_spec_init(const Prob& p, float* lam, cudaStream_t st);
// V_fm split sums on the tensor cores (and y~), grid (ceil(F / bins per CTA), S).
// tl: tensor map of lambda from scm_tensor_map, or null (per-row copies or plain loads)
cudaError_t launch_scm_tc(int maxm, const Prob& p, int S, int span, const CUtensorMap* tl, cudaStream_t st);
bool scm_tensor_map(int maxm, const Prob& p, CUtensorMap* tl);
int scm_bins_per_cta(int maxm);
int scm_frames_per_stage(int maxm);
int scm_smem(int maxm, int N);             // dynamic shared memory of k_scm_tc for N sources
cudaError_t scm_prepare(int maxm, int N);  // allow that much shared memory
int scm_occupancy(int maxm, int N);        // resident k_scm_tc CTAs per SM
// tensor-core g~ update (N padded to np sources; np = 0: N unsupported)
int gtc_np(int maxm, int N);
// tx, tl: tensor maps of x~ and lambda from gtc_tensor_maps, or null (the kernel's threads
// then load the inputs)
cudaError_t launch_g_tc(int maxm, int np, const Prob& p, int S, int span, unsigned ctr, const CUtensorMap* tx,
                        const CUtensorMap* tl, cudaStream_t st);
bool gtc_tensor_maps(int maxm, const Prob& p, CUtensorMap* tx, CUtensorMap* tl);
cudaError_t gtc_prepare(int maxm, int np, int N);
int gtc_occupancy(int maxm, int np, int N);
int gtc_smem(int maxm, int np, int N);
int gtc_bins_per_cta(int maxm);
int gtc_frames_per_stage();
cudaError_t launch_apply(float* fac, const float* C, int S, int N, int K, int own, unsigned* status,
                         cudaStream_t st);

// FastMNMF-DP (fm_dp.cu): the deep-prior speech source (source 0) and NMF noise sources
// (1..N-1) around the unconstrained-model context's lambda, g~, Q and x~.
struct DpArgs {
  Prob p;                        // the inner context's problem (X, G, Qf, xt, status, ...)
  float* lam = nullptr;          // [N][F][T]
  float* u = nullptr;            // [F]
  float* v = nullptr;            // [T]
  float* Z = nullptr;            // [T][D]
  float* R = nullptr;            // [F][T] decoder output of Z
  float* Wn = nullptr;           // [N-1][K][F]
  float* Hn = nullptr;           // [N-1][K][T]
  const float* W1 = nullptr;     // [Hd][D]
  const float* b1 = nullptr;     // [Hd]
  const float* W2 = nullptr;     // [F][Hd]
  const float* b2 = nullptr;     // [F]
  int D = 0, Hd = 0, K = 0;
  const float* xi = nullptr;     // [S][T][D] draws of this iteration
  const float* logu = nullptr;   // [S][T]
  int S = 0;
  float sqrt_eps = 0.f;
  unsigned long long* n_acc = nullptr;  // accepted proposals (accumulated)
  float* loggamma = nullptr;     // [S][T] log gamma of every proposal, or null
  const float* nu = nullptr;     // [N][F] nu of the last normalisation (k_bin)
  int maxm = 8;
  int tb = 1;                    // frames per Metropolis cluster
};
// Launch shape of the Metropolis kernel: clusters of C CTAs (the bins split C ways), TB frames
// per cluster, FG frames per thread; C = 0 when nothing fits in `limit` bytes of shared memory.
struct DpMhPlan {
  int C = 0, TB = 0, FG = 0, threads = 0;
  size_t smem = 0;
};
DpMhPlan dp_mh_plan(int F, int T, int M, int D, int Hd, int sms, size_t limit);
cudaError_t dp_prepare(int maxm, const DpMhPlan& plan);
cudaError_t dp_launch_init(const DpArgs& a, cudaStream_t st);     // R from Z, lambda of every source
cudaError_t dp_launch_mh(const DpArgs& a, const DpMhPlan& plan, cudaStream_t st);  // S proposals per frame
cudaError_t dp_launch_fsweep(const DpArgs& a, int mode, cudaStream_t st);  // per bin: u (0) or noise W (1)
cudaError_t dp_launch_tsweep(const DpArgs& a, int mode, cudaStream_t st);  // per frame: v (0) or noise H (1)
cudaError_t dp_launch_norm(const DpArgs& a, cudaStream_t st);     // nu into u, W; mu into v, H

// Largest dynamic shared memory of the IP kernel's prefetch (X and y~ rows, g~, W of a bin):
// small enough that four or more IP CTAs stay resident per SM.
constexpr int kIpPrefetchMax = 40 * 1024;

// Sets the calling thread's message returned by fmnmf_last_error(NULL).
void set_thread_error(const char* msg);

}  // namespace fm
