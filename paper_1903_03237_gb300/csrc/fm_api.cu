// Host runtime of libfastmnmf.so: the C ABI declared in include/fastmnmf.h.
//
// A context owns one device arena (a single cudaMalloc) holding the mixture, the state
// and the scratch of the split reductions, the tiling of every launch, and a cache of
// CUDA graphs (one per chunk length of fmnmf_iterate) so that an iteration costs one
// graph launch instead of five kernel launches from the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fastmnmf.h"
#include "fm_fused.cuh"
#include "fm_gemm.cuh"
#include "fm_kernels.cuh"
#include "fm_launch.h"

namespace {

using namespace fm;

thread_local std::string g_thread_err;

constexpr int kMaxChunk = 100;          // iterations per captured graph
constexpr int kSmemTarget = 72 * 1024;   // bytes per CTA aimed for (three CTAs per SM)
constexpr int kSmemMax = 220 * 1024;     // hard ceiling (227 KB per CTA on sm_103a)

const char* kKindNames[KK_COUNT] = {"w_update", "h_update", "g_update", "scm", "xt_loglik",
                                    "prep_q", "wiener", "ip", "gemm_lambda", "gemm_w", "gemm_h",
                                    "pr", "apply", "bin", "hgemm"};

// One tensor-core GEMM of the mixed form, planned once per context.
struct GemmPlan {
  GemmArgs g{};
  dim3 grid;
  int nt = 128;
};

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;  // (kind, start/end)
  int launches = 0;
  bool unharvested = false;  // timing graphs: events hold a launch not yet accumulated
};

}  // namespace

struct fmnmf_ctx {
  int F = 0, T = 0, M = 0, N = 0, K = 0, maxm = 0;
  fmnmf_opts opts{};
  cudaStream_t st = nullptr;
  bool own_stream = false;
  Prob p{};
  void* arena = nullptr;
  size_t arena_bytes = 0;
  Geom gW{}, gH{}, gG{}, gY{}, gS{};
  size_t smW = 0, smH = 0, smG = 0, smY = 0, smS = 0;
  int n_pt_blocks = 0, n_mu_blocks = 0;
  size_t ipSmem = 0;  // the IP kernel's prefetch buffers (0: none)
  bool fusedPR = false;  // the kernel that forms x~ also forms P, R of the next W update
  // fused FP32 schedule (k_hgemm + k_bin per iteration) and the unconstrained source model
  bool fused = false, free_model = false;
  int hgS = 1, hgSpan = 32;        // H GEMM: bin splits (one cluster per tile) and bins per split
  size_t binSm = 0;                // k_bin's dynamic shared memory
  bool prsm = false;               // k_bin keeps the W update's P, R in shared memory
  bool lamsm = false;              // k_bin keeps the bin's lambda in shared memory
  float* lam0 = nullptr;           // restart copy of lambda (unconstrained model)
  unsigned ctrW = 0, ctrH = 0, ctrG = 0, ctrY = 0, ctrLL = 0;
  // copy of the state set by the last init / reset / set_state (for fmnmf_restart)
  float* W0 = nullptr;
  float* H0 = nullptr;
  float* G0 = nullptr;
  float4* Q0 = nullptr;
  // mixed-precision form
  bool mixed = false, tf32 = false;
  float* lam = nullptr;   // [N][F][T]
  float* PR = nullptr;    // [2][N][F][T]
  float* Cg = nullptr;    // split GEMM sums
  GemmPlan gpW, gpH, gpL;
  int scmS = 1, scmSpan = 64;  // tensor-core V_fm: T splits and frames per split
  int gtcNP = 0, gtcS = 1, gtcSpan = 16;  // tensor-core g~ update (NP = 0: the CUDA-core sweep)
  bool gtcTma = false;                     // tensor maps of x~ and lambda for its inputs
  alignas(64) CUtensorMap gtcTmX, gtcTmL;
  bool scmTma = false;                     // tensor map of lambda for the V_fm kernel
  alignas(64) CUtensorMap scmTmL;
  // launch shapes: the split counts plan() chose for the tunable launches, and the tuner's
  // scales of them (<= 1: buffers are sized for the planned counts)
  int caps[4] = {0, 0, 0, 0};
  int baseS[8] = {1, 1, 1, 1, 1, 1, 1, 1};
  float tscale[8] = {1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f};
  int sms = 0;
  std::map<std::pair<int, unsigned>, GraphEntry> graphs;  // (chunk, timing mask) -> graph
  std::string err;
  unsigned timing = 0;  // bit i: bracket launches of kernel class i with events
  double ms[KK_COUNT] = {0};
  long long cnt[KK_COUNT] = {0};
  long long launches = 0;
  // events for timed direct launches (separate)
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  std::vector<cudaEvent_t> evpool;
};

// A batch: several contexts iterated by one CUDA graph with one branch per context.
struct fmnmf_batch {
  std::vector<fmnmf_ctx*> ctxs;
  cudaStream_t st = nullptr;  // origin stream: fork and join point of the branches
  std::map<int, cudaGraphExec_t> graphs;  // chunk length -> executable graph
  std::map<int, long long> graph_launches;
  std::vector<cudaEvent_t> events;
  std::string err;
};

namespace {

fmnmf_status set_err(fmnmf_ctx* c, fmnmf_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf; else g_thread_err = buf;
  return s;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return set_err(ctx, FMNMF_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));   \
  } while (0)

int bucket(int M) { return M <= 2 ? 2 : (M <= 4 ? 4 : 8); }

cudaError_t launch(fmnmf_ctx* c, KernelKind k, const LaunchArgs& a) {
  c->launches++;
  switch (c->maxm) {
    case 2: return launch_m2(k, a);
    case 4: return launch_m4(k, a);
    default: return launch_m8(k, a);
  }
}

int occupancy(int maxm, KernelKind k, size_t smem) {
  switch (maxm) {
    case 2: return occupancy_m2(k, smem);
    case 4: return occupancy_m4(k, smem);
    default: return occupancy_m8(k, smem);
  }
}

// The dynamic shared-memory limit is a property of each kernel function (per device), shared
// by every context: it is only ever raised, so that a context that needs less never lowers it
// under another's launches.
cudaError_t configure(int maxm, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, int> set_to;  // (device, bucket) -> bytes
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  int& cur = set_to[{dev, maxm}];
  if (bytes <= cur) return cudaSuccess;
  switch (maxm) {
    case 2: e = configure_m2(bytes); break;
    case 4: e = configure_m4(bytes); break;
    default: e = configure_m8(bytes); break;
  }
  if (e == cudaSuccess) cur = bytes;
  return e;
}

// Tiling of a sweep over an own extent SO (tiles of kOT) and an inner extent SI split
// S ways so that the grid fills the `slots` CTAs the device holds at once (one wave);
// sub-chunks of at most ic_cap.
Geom make_geom(int SO, int SI, int ic_cap, int slots) {
  Geom g;
  g.n_own_tiles = (SO + kOT - 1) / kOT;
  int S = std::max(1, slots / g.n_own_tiles);
  S = std::min(S, (SI + 3) / 4);
  int span = (SI + S - 1) / S;
  span = (span + 3) & ~3;
  g.S = (SI + span - 1) / span;
  g.span = span;
  g.IC = std::min(ic_cap, span);
  g.ICP = g.IC + 4;
  return g;
}

// The same tiling with a given number of inner splits.
Geom make_geom_S(int SO, int SI, int ic_cap, int S) {
  Geom g;
  g.n_own_tiles = (SO + kOT - 1) / kOT;
  S = std::max(1, std::min(S, (SI + 3) / 4));
  int span = (SI + S - 1) / S;
  span = (span + 3) & ~3;
  g.S = (SI + span - 1) / span;
  g.span = span;
  g.IC = std::min(ic_cap, span);
  g.ICP = g.IC + 4;
  return g;
}

// Tunable launches: the inner split counts of the sweeps, the tensor-core V_fm and g~
// kernels and the split-K GEMMs of the W and H sums.
enum { TU_W = 0, TU_H, TU_G, TU_Y, TU_SCM, TU_GTC, TU_GEMM_W, TU_GEMM_H, TU_COUNT };

// Largest sub-chunk (multiple of 4, <= 256) whose shared memory fits `limit` bytes.
int ic_cap_for(int mode, int N, int K, int M, int maxm, int limit, bool lam_mem = false) {
  for (int ic = 256; ic >= 4; ic -= 4) {
    size_t bytes = (size_t)tile_smem(mode, N, K, M, maxm, ic, lam_mem).total * 4;
    if (bytes <= (size_t)limit) return ic;
  }
  return 0;
}

size_t smem_bytes(int mode, int N, int K, int M, int maxm, int ic, bool lam_mem = false) {
  size_t b = (size_t)tile_smem(mode, N, K, M, maxm, ic, lam_mem).total * 4;
  return b;
}

// k_separate: Q and Q^-1 of the tile's bins, g~; unless lambda is read from memory, the W
// tile, an H chunk and the lambda chunk.
size_t sep_smem_bytes(int N, int K, int M, int maxm, int ic, bool lam_mem = false) {
  const int NK = N * K, ICP = ic + 4;
  size_t fl = (((size_t)N * kOT * M + 3) & ~(size_t)3);
  if (!lam_mem) fl += (size_t)NK * kOT + (size_t)NK * ICP + (size_t)N * kOT * ICP;
  return fl * 4 + 2 * (size_t)kOT * maxm * maxm * sizeof(float2);
}

// Mixtures of at most this many frames form x~ and the log-likelihood inside the IP kernel
// (see enqueue_tail).
constexpr int kFuseXtFrames = 1024;

void apply_fused_shape(fmnmf_ctx* c);

fmnmf_status plan(fmnmf_ctx* ctx) {
  const int F = ctx->F, T = ctx->T, M = ctx->M, N = ctx->N, K = ctx->K, mx = ctx->maxm;
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int caps[4];
  // the mixed form (and the unconstrained source model) reads lambda in the g~ and y~
  // sweeps: no factor tiles there
  const bool lam_ctx = ctx->mixed || ctx->free_model;
  auto lm = [&](int mode) { return lam_ctx && (mode == MODE_G || mode == MODE_Y); };
  for (int mode = 0; mode < 4; ++mode) {
    int cap = ic_cap_for(mode, N, K, M, mx, kSmemTarget, lm(mode));
    if (cap == 0) cap = ic_cap_for(mode, N, K, M, mx, kSmemMax, lm(mode));
    if (cap == 0) return set_err(ctx, FMNMF_EINVAL, "N*K = %d too large for the shared-memory tiles", N * K);
    caps[mode] = cap;
  }
  size_t mx_cap_smem = 48 * 1024;
  for (int mode = 0; mode < 4; ++mode)
    mx_cap_smem = std::max(mx_cap_smem, smem_bytes(mode, N, K, M, mx, caps[mode], lm(mode)));
  CK(configure(mx, (int)mx_cap_smem));
  const KernelKind kinds[4] = {KK_W, KK_H, KK_G, KK_Y};
  auto slots = [&](int mode) {
    return sms * occupancy(mx, kinds[mode], smem_bytes(mode, N, K, M, mx, caps[mode], lm(mode)));
  };
  ctx->gW = make_geom(F, T, caps[MODE_W], slots(MODE_W));
  ctx->gH = make_geom(T, F, caps[MODE_H], slots(MODE_H));
  ctx->gG = make_geom(F, T, caps[MODE_G], slots(MODE_G));
  ctx->gY = make_geom(F, T, caps[MODE_Y], slots(MODE_Y));
  ctx->smW = smem_bytes(MODE_W, N, K, M, mx, ctx->gW.IC);
  ctx->smH = smem_bytes(MODE_H, N, K, M, mx, ctx->gH.IC);
  ctx->smG = smem_bytes(MODE_G, N, K, M, mx, ctx->gG.IC, lm(MODE_G));
  ctx->smY = smem_bytes(MODE_Y, N, K, M, mx, ctx->gY.IC, lm(MODE_Y));
  // the Wiener filter reads the materialised lambda in the mixed form and the free model
  const bool sep_lm = lam_ctx;
  int sep_cap = 0;
  for (int ic = 256; ic >= 4; ic -= 4)
    if (sep_smem_bytes(N, K, M, mx, ic, sep_lm) <= (size_t)kSmemTarget) { sep_cap = ic; break; }
  if (sep_cap == 0)
    for (int ic = 256; ic >= 4; ic -= 4)
      if (sep_smem_bytes(N, K, M, mx, ic, sep_lm) <= (size_t)kSmemMax) { sep_cap = ic; break; }
  if (sep_cap == 0) return set_err(ctx, FMNMF_EINVAL, "N*K too large for the Wiener tiles");
  mx_cap_smem = std::max(mx_cap_smem, sep_smem_bytes(N, K, M, mx, sep_cap, sep_lm));
  CK(configure(mx, (int)mx_cap_smem));
  ctx->gS = make_geom(F, T, sep_cap, sms * occupancy(mx, KK_SEP, sep_smem_bytes(N, K, M, mx, sep_cap, sep_lm)));
  ctx->smS = sep_smem_bytes(N, K, M, mx, ctx->gS.IC, sep_lm);
  ctx->sms = sms;
  if (ctx->mixed) {
    CK(configure_gemm());
    auto nt_for = [](int n) { return n <= 16 ? 16 : n <= 32 ? 32 : n <= 64 ? 64 : 128; };
    auto plan_gemm = [&](GemmPlan& gp, int Mr, int Nc, int Kd, int batch, int nt, bool allow_split) {
      gp.nt = nt;
      gp.g.Mr = Mr; gp.g.Nc = Nc; gp.g.Kd = Kd; gp.g.batch = batch;
      const int mt = (Mr + 127) / 128, ntl = (Nc + nt - 1) / nt;
      const int kchunks = (Kd + kGemmKc - 1) / kGemmKc;
      int S = 1;
      if (allow_split) S = std::max(1, std::min(kchunks, (2 * sms + mt * ntl * batch - 1) / (mt * ntl * batch)));
      // a TMEM accumulator sums its split sequentially in FP32: at most 512 terms per split
      // (the splits are then summed in a fixed order), which bounds the rounding growth
      S = std::max(S, (Kd + 511) / 512);
      const int kspan = ((kchunks + S - 1) / S) * kGemmKc;
      S = (Kd + kspan - 1) / kspan;
      gp.g.ksplit = S; gp.g.kspan = kspan;
      gp.grid = dim3(mt, ntl, batch * S);
    };
    plan_gemm(ctx->gpW, F, K, T, 2 * N, nt_for(K), true);
    plan_gemm(ctx->gpH, T, K, F, 2 * N, nt_for(K), true);
    // lambda: the widest column tile that still gives about two waves of CTAs
    int ntL = 128;
    while (ntL > 32 && (long long)((F + 127) / 128) * ((T + ntL - 1) / ntL) * N < 2LL * sms) ntL /= 2;
    plan_gemm(ctx->gpL, F, T, K, N, ntL, false);
    // V_fm: bin groups x T splits.  Enough splits for two waves, then the split count (up
    // to twice that) whose last wave is fullest; spans are whole stages.
    const int nb = (F + scm_bins_per_cta(mx) - 1) / scm_bins_per_cta(mx);
    if (scm_smem(mx, N) > 227 * 1024)
      return set_err(ctx, FMNMF_EINVAL, "N=%d is too large for the mixed-precision form (use FP32)", N);
    CK(scm_prepare(mx, N));
    const int kc = scm_frames_per_stage(mx);
    const int nst = (T + kc - 1) / kc;
    const int slots = sms * scm_occupancy(mx, N);
    const int S0 = std::max(1, std::min(nst, (2 * slots + nb - 1) / nb));
    int best = S0;
    double best_fill = 0.0;
    for (int S = S0; S <= std::min(nst, 2 * S0); ++S) {
      const double w = (double)nb * S / slots;
      const double fill = w / std::ceil(w);
      if (fill > best_fill + 1e-9) { best_fill = fill; best = S; }
    }
    ctx->scmSpan = ((nst + best - 1) / best) * kc;
    ctx->scmS = (T + ctx->scmSpan - 1) / ctx->scmSpan;
    // g~ update: the same split choice for its bin groups
    ctx->gtcNP = gtc_np(mx, N);
    if (ctx->gtcNP > 0 && gtc_smem(mx, ctx->gtcNP, N) <= 227 * 1024) {
      CK(gtc_prepare(mx, ctx->gtcNP, N));
      const int gnb = (F + gtc_bins_per_cta(mx) - 1) / gtc_bins_per_cta(mx);
      const int gkc = gtc_frames_per_stage();
      const int gst = (T + gkc - 1) / gkc;
      const int gslots = sms * gtc_occupancy(mx, ctx->gtcNP, N);
      const int G0 = std::max(1, std::min(gst, (2 * gslots + gnb - 1) / gnb));
      int gbest = G0;
      double gfill = 0.0;
      for (int S = G0; S <= std::min(gst, 2 * G0); ++S) {
        const double w = (double)gnb * S / gslots;
        const double fill = w / std::ceil(w);
        if (fill > gfill + 1e-9) { gfill = fill; gbest = S; }
      }
      ctx->gtcSpan = ((gst + gbest - 1) / gbest) * gkc;
      ctx->gtcS = (T + ctx->gtcSpan - 1) / ctx->gtcSpan;
    } else {
      ctx->gtcNP = 0;
    }
  }
  ctx->n_pt_blocks = (int)(((size_t)F * T + kThreads * kPtsPerThread - 1) / (kThreads * kPtsPerThread));
  ctx->n_mu_blocks = N * K;  // one CTA per (n, k) row
  {
    // the IP kernel prefetches the bin's X and y~ rows (when it forms x~), g~ and W
    const size_t tm = (size_t)T * M;
    const size_t pfb = (2 * tm + ((tm + 3) & ~(size_t)3) + (((size_t)N * M + 3) & ~(size_t)3) + (size_t)N * K) * 4;
    ctx->ipSmem = (T <= kFuseXtFrames && pfb <= (size_t)kIpPrefetchMax) ? pfb : 0;
  }
  {
    // mixed form with a W update to feed: the kernel that forms x~ at the end of an
    // iteration (the IP kernel for short mixtures, else k_xt_ll) forms P, R
    ctx->fusedPR = ctx->mixed && (ctx->opts.update_mask & FMNMF_UPDATE_W);
  }
  {
    // fused schedule (FP32): per-bin kernel + H kernel, when its pair limits and shared
    // memory allow; the unconstrained source model runs only there
    const int Kf = ctx->free_model ? 1 : K;
    const size_t bsm = (size_t)bin_smem(N, Kf, mx).total * 4;
    bool ok = !ctx->mixed && N * M <= kFuMaxNM && bsm <= (size_t)kSmemMax;
    // H GEMM: bin splits chosen per shape (apply_fused_shape), one thread-block cluster per tile
    const int sched = ctx->opts.schedule;
    if (ctx->free_model && !ok)
      return set_err(ctx, FMNMF_EINVAL, "the unconstrained source model needs the fused FP32 schedule (N*M <= %d)",
                     kFuMaxNM);
    if (sched == FMNMF_SCHED_FUSED && !ok)
      return set_err(ctx, FMNMF_EINVAL, "fused schedule not available for this shape/precision (FP32, N*M <= %d, "
                     "per-bin tiles within shared memory)", kFuMaxNM);
    ctx->fused = ok && (ctx->free_model || sched != FMNMF_SCHED_SWEEP);
    if (ctx->fused) {
      ctx->binSm = bsm;
      mx_cap_smem = std::max(mx_cap_smem, ctx->binSm);
      // the W update's P, R and the bin's lambda in shared memory, when they fit without
      // costing a resident CTA (the first of these layouts that keeps the occupancy)
      if (!ctx->free_model) {
        auto occ = [&](size_t b) {
          switch (mx) {
            case 2: return occupancy_fused_m2(KK_BIN, b);
            case 4: return occupancy_fused_m4(KK_BIN, b);
            default: return occupancy_fused_m8(KK_BIN, b);
          }
        };
        const size_t nt = (size_t)N * T;
        struct Cand { bool pr, lam; };
        const Cand cands[3] = {{true, true}, {true, false}, {false, true}};
        for (const Cand& cd : cands) {
          if ((cd.pr && 2 * nt * 4 > 32 * 1024) || (cd.lam && nt * 4 > 16 * 1024)) continue;
          const size_t b = 4 * (cd.lam ? (size_t)bin_smem_lam_offset(N, Kf, mx, T, cd.pr) + nt
                                       : (size_t)bin_smem_pr_offset(N, Kf, mx) + 2 * nt);
          if (b > (size_t)kSmemMax) continue;
          CK(configure(mx, (int)std::max(mx_cap_smem, b)));
          const int o0 = occ(bsm), o1 = occ(b);
          if (o1 >= o0 && o1 > 0) {
            ctx->prsm = cd.pr;
            ctx->lamsm = cd.lam;
            ctx->binSm = b;
            mx_cap_smem = std::max(mx_cap_smem, b);
            break;
          }
        }
      }
      CK(configure(mx, (int)mx_cap_smem));
    }
  }
  for (int mode = 0; mode < 4; ++mode) ctx->caps[mode] = caps[mode];
  const int base[TU_COUNT] = {ctx->gW.S, ctx->gH.S, ctx->gG.S, ctx->gY.S, ctx->scmS, ctx->gtcS,
                              ctx->mixed ? ctx->gpW.g.ksplit : 1, ctx->mixed ? ctx->gpH.g.ksplit : 1};
  for (int t = 0; t < TU_COUNT; ++t) { ctx->baseS[t] = base[t]; ctx->tscale[t] = 1.f; }
  apply_fused_shape(ctx);
  return FMNMF_OK;
}

// The fused schedule's H GEMM: S bin splits per tile (the CTAs of one cluster), the largest
// even S (at most the portable cluster size 8) that keeps the grid within two CTAs per SM,
// else 1; and the bins per split.  Even sizes: on the paper-scale mixture (40 tiles) S = 6
// measured 1 % faster per iteration than 8, and 7 2 % slower than 6.
void apply_fused_shape(fmnmf_ctx* c) {
  if (!c->fused) return;
  const long long tiles = (long long)c->N * ((c->K + kHgKT - 1) / kHgKT) * ((c->T + kHgTT - 1) / kHgTT);
  const long long sms = c->sms > 0 ? c->sms : 1;
  long long S = std::min((long long)kHgMaxS, 2 * sms / std::max(1LL, tiles));
  S = S >= 2 ? S & ~1LL : 1;
  c->hgS = (int)S;
  c->hgSpan = (c->F + c->hgS - 1) / c->hgS;
}

// Re-derives the tunable launch shapes from the planned split counts and the tuner's scales.
void apply_shapes(fmnmf_ctx* c) {
  const int F = c->F, T = c->T, M = c->M, N = c->N, K = c->K, mx = c->maxm;
  auto S_of = [&](int t, int smin) { return std::max(smin, (int)std::lround(c->baseS[t] * c->tscale[t])); };
  auto lm = [&](int mode) { return (c->mixed || c->free_model) && (mode == MODE_G || mode == MODE_Y); };
  c->gW = make_geom_S(F, T, c->caps[MODE_W], S_of(TU_W, 1));
  c->gH = make_geom_S(T, F, c->caps[MODE_H], S_of(TU_H, 1));
  c->gG = make_geom_S(F, T, c->caps[MODE_G], S_of(TU_G, 1));
  c->gY = make_geom_S(F, T, c->caps[MODE_Y], S_of(TU_Y, 1));
  c->smW = smem_bytes(MODE_W, N, K, M, mx, c->gW.IC);
  c->smH = smem_bytes(MODE_H, N, K, M, mx, c->gH.IC);
  c->smG = smem_bytes(MODE_G, N, K, M, mx, c->gG.IC, lm(MODE_G));
  c->smY = smem_bytes(MODE_Y, N, K, M, mx, c->gY.IC, lm(MODE_Y));
  apply_fused_shape(c);
  if (!c->mixed) return;
  auto frames = [&](int S, int kc, int& span, int& outS) {
    const int nst = (T + kc - 1) / kc;
    S = std::max(1, std::min(S, nst));
    span = ((nst + S - 1) / S) * kc;
    outS = (T + span - 1) / span;
  };
  frames(S_of(TU_SCM, 1), scm_frames_per_stage(mx), c->scmSpan, c->scmS);
  if (c->gtcNP > 0) frames(S_of(TU_GTC, 1), gtc_frames_per_stage(), c->gtcSpan, c->gtcS);
  auto gemm = [&](GemmPlan& gp, int S) {
    const int kchunks = (gp.g.Kd + kGemmKc - 1) / kGemmKc;
    S = std::max(S, (gp.g.Kd + 511) / 512);  // at most 512 terms per TMEM accumulator
    const int kspan = ((kchunks + S - 1) / S) * kGemmKc;
    gp.g.ksplit = (gp.g.Kd + kspan - 1) / kspan;
    gp.g.kspan = kspan;
    gp.grid.z = (unsigned)(gp.g.batch * gp.g.ksplit);
  };
  gemm(c->gpW, S_of(TU_GEMM_W, 1));
  gemm(c->gpH, S_of(TU_GEMM_H, 1));
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Lays out (dry_run: only sizes, into ctx->arena_bytes) or allocates the context arena.
fmnmf_status allocate(fmnmf_ctx* ctx, bool dry_run = false) {
  const size_t F = ctx->F, T = ctx->T, M = ctx->M, N = ctx->N, K = ctx->K;
  const int mx = ctx->maxm;
  size_t part = 0;
  part = std::max(part, (size_t)ctx->gW.S * tile_part_floats(MODE_W, F, T, M, N, K, mx));
  part = std::max(part, (size_t)ctx->gH.S * tile_part_floats(MODE_H, F, T, M, N, K, mx));
  part = std::max(part, (size_t)ctx->gG.S * tile_part_floats(MODE_G, F, T, M, N, K, mx));
  part = std::max(part, (size_t)ctx->gY.S * tile_part_floats(MODE_Y, F, T, M, N, K, mx));
  if (ctx->mixed) part = std::max(part, (size_t)ctx->scmS * tile_part_floats(MODE_Y, F, T, M, N, K, mx));
  if (ctx->mixed && ctx->gtcNP > 0) part = std::max(part, (size_t)ctx->gtcS * tile_part_floats(MODE_G, F, T, M, N, K, mx));
  const unsigned nctr = ctx->gW.n_own_tiles + ctx->gH.n_own_tiles + ctx->gG.n_own_tiles +
                        ctx->gY.n_own_tiles + 1;
  ctx->ctrW = 0;
  ctx->ctrH = ctx->ctrW + ctx->gW.n_own_tiles;
  ctx->ctrG = ctx->ctrH + ctx->gH.n_own_tiles;
  ctx->ctrY = ctx->ctrG + ctx->gG.n_own_tiles;
  ctx->ctrLL = ctx->ctrY + ctx->gY.n_own_tiles;
  struct Slot { void** dst; size_t bytes; };
  Prob& p = ctx->p;
  void* X = nullptr;
  std::vector<Slot> slots = {
      {&X, F * T * M * sizeof(float2)},
      {(void**)&p.W, N * K * F * 4},
      {(void**)&p.H, N * K * T * 4},
      {(void**)&p.G, N * F * M * 4},
      {(void**)&p.Qx, F * M * M * sizeof(float4)},
      {(void**)&p.Qix, F * M * M * sizeof(float4)},
      {(void**)&p.Qf, F * M * M * sizeof(float2)},
      {(void**)&p.Qinv, F * M * M * sizeof(float2)},
      {(void**)&p.xt, F * T * M * 4},
      {(void**)&p.yt, F * T * M * 4},
      {(void**)&p.logdet, F * 8},
      {(void**)&p.phi, F * 4},
      {(void**)&p.ll, 8},
      {(void**)&p.status, 4},
      {(void**)&p.part, part * 4},
      {(void**)&p.llpart, (size_t)std::max(ctx->n_pt_blocks, ctx->F) * 8},
      {(void**)&p.counters, (size_t)nctr * 4},
      {(void**)&ctx->W0, N * K * F * 4},
      {(void**)&ctx->H0, N * K * T * 4},
      {(void**)&ctx->G0, N * F * M * 4},
      {(void**)&ctx->Q0, F * M * M * sizeof(float4)},
  };
  if (ctx->fused) {
    slots.push_back({(void**)&ctx->lam, N * F * T * 4});
    if (!ctx->free_model) slots.push_back({(void**)&ctx->PR, 2 * N * F * T * 4});
    else slots.push_back({(void**)&ctx->lam0, N * F * T * 4});
  }
  if (ctx->mixed) {
    const size_t cg = std::max((size_t)ctx->gpW.grid.z * ctx->gpW.g.Mr * ctx->gpW.g.Nc,
                               (size_t)ctx->gpH.grid.z * ctx->gpH.g.Mr * ctx->gpH.g.Nc);
    slots.push_back({(void**)&ctx->lam, N * F * T * 4});
    slots.push_back({(void**)&ctx->PR, 2 * N * F * T * 4});
    slots.push_back({(void**)&ctx->Cg, cg * 4});
  }
  size_t total = 0;
  for (auto& s : slots) total += align256(s.bytes);
  if (dry_run) {
    ctx->arena_bytes = total;
    return FMNMF_OK;
  }
  if (ctx->opts.hbm_budget && total > ctx->opts.hbm_budget)
    return set_err(ctx, FMNMF_ENOMEM, "needs %zu bytes of device memory, budget %zu", total,
                   ctx->opts.hbm_budget);
  // stream-ordered: neither the allocation nor the release waits for other contexts' work
  cudaError_t e = cudaMallocAsync(&ctx->arena, total, ctx->st);
  if (e != cudaSuccess) return set_err(ctx, FMNMF_ENOMEM, "cudaMallocAsync(%zu): %s", total, cudaGetErrorString(e));
  ctx->arena_bytes = total;
  char* base = (char*)ctx->arena;
  for (auto& s : slots) { *s.dst = base; base += align256(s.bytes); }
  p.X = (const float2*)X;
  p.F = ctx->F; p.T = ctx->T; p.M = ctx->M; p.N = ctx->N; p.K = ctx->K;
  p.lam = nullptr;
  if (ctx->mixed) {
    const long long FT = (long long)F * T;
    GemmArgs& w = ctx->gpW.g;   // [P;R]_n (f x t) . H_n (k x t)^T
    w.A = ctx->PR; w.sAb = FT; w.sAi = T; w.sAk = 1;
    w.B = p.H; w.sBb = (long long)K * T; w.sBj = T; w.sBk = 1; w.bmodB = (int)N;
    w.C = ctx->Cg; w.sCs = 2LL * N * F * K; w.sCb = (long long)F * K; w.sCi = K; w.sCj = 1;
    w.status = p.status;
    w.wait_limit = p.wait_limit;
    GemmArgs& h = ctx->gpH.g;   // [P;R]_n^T (t x f) . W_n (k x f)^T
    h.A = ctx->PR; h.sAb = FT; h.sAi = 1; h.sAk = T;
    h.B = p.W; h.sBb = (long long)K * F; h.sBj = F; h.sBk = 1; h.bmodB = (int)N;
    h.C = ctx->Cg; h.sCs = 2LL * N * T * K; h.sCb = (long long)T * K; h.sCi = K; h.sCj = 1;
    h.status = p.status;
    h.wait_limit = p.wait_limit;
    GemmArgs& l = ctx->gpL.g;   // W_n^T (f x k) . H_n^T (t x k)^T = lambda_n (f x t)
    l.A = p.W; l.sAb = (long long)K * F; l.sAi = 1; l.sAk = F;
    l.B = p.H; l.sBb = (long long)K * T; l.sBj = 1; l.sBk = T; l.bmodB = (int)N;
    l.C = ctx->lam; l.sCs = 0; l.sCb = FT; l.sCi = T; l.sCj = 1;
    l.status = p.status;
    l.wait_limit = p.wait_limit;
    Prob q = p;
    q.lam = ctx->lam;
    if (ctx->gtcNP > 0) ctx->gtcTma = gtc_tensor_maps(ctx->maxm, q, &ctx->gtcTmX, &ctx->gtcTmL);
    ctx->scmTma = scm_tensor_map(ctx->maxm, q, &ctx->scmTmL);
  }
  CK(cudaMemsetAsync(p.counters, 0, (size_t)nctr * 4, ctx->st));
  CK(cudaMemsetAsync(p.status, 0, 4, ctx->st));
  return FMNMF_OK;
}

// ---- launches ----------------------------------------------------------------------
LaunchArgs tile_args(fmnmf_ctx* c, const Geom& g, size_t smem, int flags, unsigned ctr) {
  LaunchArgs a;
  a.p = c->p; a.g = g; a.smem = smem; a.st = c->st; a.flags = flags; a.ctr = ctr;
  a.grid = dim3(g.n_own_tiles, g.S);
  return a;
}

struct Recorder {  // brackets launches with events when timing is on (works under capture)
  fmnmf_ctx* c;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>>* out;
  cudaEvent_t take() {
    cudaEvent_t e;
    if (!c->evpool.empty()) { e = c->evpool.back(); c->evpool.pop_back(); }
    else cudaEventCreate(&e);
    return e;
  }
  cudaError_t run(KernelKind k, const LaunchArgs& a) {
    return run_fn(k, [&] { return launch(c, k, a); });
  }
  template <class Fn>
  cudaError_t run_fn(KernelKind k, Fn&& fn) {
    if (!out || !((c->timing >> (int)k) & 1u)) return fn();
    cudaEvent_t e0 = take(), e1 = take();
    // under stream capture the records must be External to become event-record nodes
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t r = cudaStreamIsCapturing(c->st, &cs);
    if (r != cudaSuccess) return r;
    const unsigned fl = (cs == cudaStreamCaptureStatusActive) ? cudaEventRecordExternal : cudaEventRecordDefault;
    if ((r = cudaEventRecordWithFlags(e0, c->st, fl)) != cudaSuccess) return r;
    if ((r = fn()) != cudaSuccess) return r;
    if ((r = cudaEventRecordWithFlags(e1, c->st, fl)) != cudaSuccess) return r;
    out->push_back({(int)k, {e0, e1}});
    return cudaSuccess;
  }
};

cudaError_t enqueue_mixed_iteration(fmnmf_ctx* c, Recorder& rec, bool last);

// The end of an iteration.  With a Q update or normalisation and up to kFuseXtFrames
// frames, the IP kernel also forms x~ and the log-likelihood of each bin right after the
// bin's update (one launch instead of two: the short mixtures are launch-latency bound),
// then the mu normalisation runs.  Longer mixtures keep the separate x~ / log-likelihood
// kernel, whose many small CTAs keep more loads in flight than one CTA per bin.
// The end of an iteration: the IP update and x~ (with the bins' log-likelihood terms), and,
// at the end of a chunk (last), the mu normalisation and the log-likelihood sum: mu rescales
// w_nk and h_nk reciprocally, which leaves lambda, every ratio of the W and H rules and the
// log-likelihood unchanged, so it commutes with the updates and is applied once per chunk,
// as in the fused schedule; only the last iteration's log-likelihood is summed.
cudaError_t enqueue_tail(fmnmf_ctx* c, Recorder& rec, int yflags, int ipS, int norm, bool last) {
  cudaError_t e;
  if (yflags && c->T > kFuseXtFrames) {
    LaunchArgs a;
    a.p = c->p; a.st = c->st; a.flags = yflags; a.S = ipS;
    a.grid = dim3(c->F);
    a.xt_mode = 0;
    if ((e = rec.run(KK_IP, a)) != cudaSuccess) return e;
    LaunchArgs x;
    x.p = c->p; x.st = c->st; x.ctr = c->ctrLL;
    x.n_pt_blocks = c->n_pt_blocks;
    x.apply_phi = 1;
    x.do_mu = (norm && last) ? 1 : 0;
    x.pr = c->fusedPR ? c->PR : nullptr;
    x.grid = dim3(c->n_pt_blocks + (x.do_mu ? c->n_mu_blocks : 0));
    return rec.run(KK_XT, x);
  }
  if (yflags) {
    LaunchArgs a;
    a.p = c->p; a.st = c->st; a.flags = yflags; a.S = ipS;
    a.grid = dim3(c->F);
    a.xt_mode = 1; a.ctr = c->ctrLL;
    a.smem = c->ipSmem;
    a.pr = c->fusedPR ? c->PR : nullptr;
    // with the mu normalisation to follow (end of a chunk), its kernel adds up the
    // log-likelihood (a last block beside the mu blocks) and the IP kernel skips its serial
    // tail; inside a chunk the bins' terms are left for the last iteration's sum
    a.ll_tail = (!norm && last) ? 1 : 0;
    if ((e = rec.run(KK_IP, a)) != cudaSuccess) return e;
    if (!norm || !last) return cudaSuccess;
    LaunchArgs x;
    x.p = c->p; x.st = c->st; x.ctr = c->ctrLL;
    x.n_pt_blocks = 0; x.apply_phi = 0; x.do_mu = 1; x.ll_bins = 1;
    x.grid = dim3(c->n_mu_blocks + 1);
    return rec.run(KK_XT, x);
  }
  LaunchArgs x;
  x.p = c->p; x.st = c->st; x.ctr = c->ctrLL;
  x.n_pt_blocks = c->n_pt_blocks;
  x.apply_phi = 0;
  x.do_mu = 0;
  x.pr = c->fusedPR ? c->PR : nullptr;
  x.grid = dim3(c->n_pt_blocks);
  return rec.run(KK_XT, x);
}

cudaError_t enqueue_iteration(fmnmf_ctx* c, Recorder& rec, bool last) {
  if (c->mixed) return enqueue_mixed_iteration(c, rec, last);
  const unsigned mask = c->opts.update_mask;
  const int norm = c->opts.normalise ? FLAG_NORMALISE : 0;
  cudaError_t e;
  if (mask & FMNMF_UPDATE_W)
    if ((e = rec.run(KK_W, tile_args(c, c->gW, c->smW, 0, c->ctrW))) != cudaSuccess) return e;
  if (mask & FMNMF_UPDATE_H)
    if ((e = rec.run(KK_H, tile_args(c, c->gH, c->smH, 0, c->ctrH))) != cudaSuccess) return e;
  if (mask & FMNMF_UPDATE_G)
    if ((e = rec.run(KK_G, tile_args(c, c->gG, c->smG, FLAG_UPDATE, c->ctrG))) != cudaSuccess) return e;
  const int yflags = norm | ((mask & FMNMF_UPDATE_Q) ? FLAG_DO_V : 0);
  if ((e = rec.run(KK_Y, tile_args(c, c->gY, c->smY, yflags, c->ctrY))) != cudaSuccess) return e;
  return enqueue_tail(c, rec, yflags, c->gY.S, norm, last);
}

// The mixed-precision iteration: tensor-core GEMMs for lambda and the W / H sums.
cudaError_t enqueue_mixed_iteration(fmnmf_ctx* c, Recorder& rec, bool last) {
  const unsigned mask = c->opts.update_mask;
  const int norm = c->opts.normalise ? FLAG_NORMALISE : 0;
  cudaError_t e;
  auto gemm = [&](KernelKind k, const GemmPlan& gp) {
    return rec.run_fn(k, [&] { c->launches++; return launch_gemm(gp.g, c->tf32, gp.nt, gp.grid, c->st); });
  };
  auto pr = [&](int mode) {
    Prob q = c->p;
    q.lam = c->lam;
    return rec.run_fn(KK_PR, [&] { c->launches++; return launch_pr(c->maxm, q, c->PR, mode, c->st); });
  };
  auto apply = [&](float* fac, int S, int own) {
    return rec.run_fn(KK_APPLY, [&] {
      c->launches++;
      return launch_apply(fac, c->Cg, S, c->N, c->K, own, c->p.status, c->st);
    });
  };
  if (mask & FMNMF_UPDATE_W) {
    // P, R of the W update: formed by the previous iteration's IP kernel (or by the state
    // refresh) when fusedPR is set
    if (!c->fusedPR && (e = pr(0)) != cudaSuccess) return e;
    if ((e = gemm(KK_GW, c->gpW)) != cudaSuccess) return e;
    if ((e = apply(c->p.W, c->gpW.g.ksplit, c->F)) != cudaSuccess) return e;
  }
  if (mask & FMNMF_UPDATE_H) {
    if ((e = gemm(KK_GL, c->gpL)) != cudaSuccess) return e;
    if ((e = pr(1)) != cudaSuccess) return e;
    if ((e = gemm(KK_GH, c->gpH)) != cudaSuccess) return e;
    if ((e = apply(c->p.H, c->gpH.g.ksplit, c->T)) != cudaSuccess) return e;
  }
  if ((e = gemm(KK_GL, c->gpL)) != cudaSuccess) return e;
  if (mask & FMNMF_UPDATE_G) {
    if (c->gtcNP > 0) {
      Prob q = c->p;
      q.lam = c->lam;
      if ((e = rec.run_fn(KK_G, [&] {
             c->launches++;
             return launch_g_tc(c->maxm, c->gtcNP, q, c->gtcS, c->gtcSpan, c->ctrG, c->gtcTma ? &c->gtcTmX : nullptr,
                                c->gtcTma ? &c->gtcTmL : nullptr, c->st);
           })) != cudaSuccess)
        return e;
    } else {
      LaunchArgs a = tile_args(c, c->gG, c->smG, FLAG_UPDATE | FLAG_LAM_MEM, c->ctrG);
      a.p.lam = c->lam;
      if ((e = rec.run(KK_G, a)) != cudaSuccess) return e;
    }
  }
  const int yflags = norm | ((mask & FMNMF_UPDATE_Q) ? FLAG_DO_V : 0);
  int ipS = c->gY.S;
  if (mask & FMNMF_UPDATE_Q) {
    // y~ and the V_fm split sums on the tensor cores
    Prob q = c->p;
    q.lam = c->lam;
    // V_fm in split BF16 in either mixed form: single BF16 or TF32 operands miss the 1e-3 bar
    if ((e = rec.run_fn(KK_Y, [&] { c->launches++; return launch_scm_tc(c->maxm, q, c->scmS, c->scmSpan, c->scmTma ? &c->scmTmL : nullptr, c->st); })) != cudaSuccess)
      return e;
    ipS = c->scmS;
  } else {
    LaunchArgs a = tile_args(c, c->gY, c->smY, yflags | FLAG_LAM_MEM, c->ctrY);
    a.p.lam = c->lam;
    if ((e = rec.run(KK_Y, a)) != cudaSuccess) return e;
  }
  return enqueue_tail(c, rec, yflags, ipS, norm, last);
}

LaunchArgs hgemm_args(fmnmf_ctx* c) {
  LaunchArgs a;
  a.p = c->p; a.st = c->st; a.pr = c->PR;
  a.g.S = c->hgS; a.g.span = c->hgSpan;
  a.grid = dim3((c->T + kHgTT - 1) / kHgTT, (c->K + kHgKT - 1) / kHgKT, c->N * c->hgS);
  return a;
}

// A run of n iterations in the fused FP32 schedule (fm_fused.cuh):
//   k_bin (prologue)               lambda of the bin, the first W update (Eq. 23) and P, R of
//                                  the first H update, when W or H is updated
//   n times: k_hgemm, k_bin        the H update (Eq. 24); per bin lambda, the g~ update,
//                                  V_fm + IP, normalisation, x~, the terms of Eq. 17 and, but
//                                  in the last iteration, the next W update and the next H
//                                  update's P, R
//   k_xt_ll (mu + log-likelihood)  the mu normalisation and the sum of Eq. 17
// With the unconstrained source model k_bin starts with the lambda update of Eq. 22 and there
// is no H update.
cudaError_t enqueue_fused_chunk(fmnmf_ctx* c, Recorder& rec, int n) {
  const unsigned mask = c->opts.update_mask;
  const bool norm = c->opts.normalise != 0;
  const bool fm = c->free_model;
  const bool upW = !fm && (mask & FMNMF_UPDATE_W), upH = !fm && (mask & FMNMF_UPDATE_H);
  cudaError_t e;
  auto bin = [&](int flags) {
    LaunchArgs a;
    a.p = c->p; a.st = c->st; a.grid = dim3(c->F); a.smem = c->binSm; a.flags = flags;
    a.lam = c->lam; a.pr = c->PR;
    return rec.run(KK_BIN, a);
  };
  const int lam0 = fm ? 0 : (FU_LAM0 | (c->prsm ? FU_PRSM : 0) | (c->lamsm ? FU_LAMSM : 0));
  const int base = ((mask & FMNMF_UPDATE_G) ? FU_G : 0) | ((mask & FMNMF_UPDATE_Q) ? FU_Q : 0) |
                   (norm ? FU_NORM : 0) | (fm ? FU_FREE : 0) | ((fm && (mask & FMNMF_UPDATE_W)) ? FU_LAM : 0) | lam0;
  if ((upW || upH) && (e = bin(FU_WONLY | lam0 | (upW ? FU_W : 0) | (upH ? FU_PH : 0))) != cudaSuccess) return e;
  for (int i = 0; i < n; ++i) {
    if (upH && (e = rec.run(KK_HGEMM, hgemm_args(c))) != cudaSuccess) return e;
    const bool last = i == n - 1;
    int fl = base;
    if (upW && !last) fl |= FU_W;
    if (upH && !last) fl |= FU_PH;
    // lambda * nu in memory: the unconstrained model's state, or the next H update's lambda
    // when W is not updated
    if (fm || (upH && !upW && !last)) fl |= FU_LAMWB;
    if ((e = bin(fl)) != cudaSuccess) return e;
  }
  LaunchArgs x;
  x.p = c->p; x.st = c->st; x.ctr = c->ctrLL;
  x.n_pt_blocks = 0; x.apply_phi = 0; x.do_mu = (norm && !fm) ? 1 : 0; x.ll_bins = 1;
  x.grid = dim3((x.do_mu ? c->n_mu_blocks : 0) + 1);
  return rec.run(KK_XT, x);
}

// n iterations of a context, enqueued on its stream (under capture).
cudaError_t enqueue_chunk(fmnmf_ctx* c, Recorder& rec, int n) {
  if (c->fused) return enqueue_fused_chunk(c, rec, n);
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < n && e == cudaSuccess; ++i) e = enqueue_iteration(c, rec, i == n - 1);
  return e;
}

void sync_wait_limit(fmnmf_ctx* ctx);

// x~, y~, log-det and log-likelihood of the state currently on the device.
fmnmf_status refresh_state(fmnmf_ctx* ctx) {
  sync_wait_limit(ctx);
  LaunchArgs a;
  a.p = ctx->p; a.st = ctx->st;
  a.grid = dim3((ctx->F + 7) / 8);
  CK(launch(ctx, KK_PREP, a));
  if (ctx->mixed) {
    // lambda on the tensor cores, then y~ from it (the launch geometry of the mixed form)
    ctx->launches++;
    CK(launch_gemm(ctx->gpL.g, ctx->tf32, ctx->gpL.nt, ctx->gpL.grid, ctx->st));
    LaunchArgs y = tile_args(ctx, ctx->gY, ctx->smY, FLAG_LAM_MEM, ctx->ctrY);
    y.p.lam = ctx->lam;
    CK(launch(ctx, KK_Y, y));
  } else if (ctx->free_model) {
    // y~ from the lambda state
    LaunchArgs y = tile_args(ctx, ctx->gY, ctx->smY, FLAG_LAM_MEM, ctx->ctrY);
    y.p.lam = ctx->lam;
    CK(launch(ctx, KK_Y, y));
  } else {
    CK(launch(ctx, KK_Y, tile_args(ctx, ctx->gY, ctx->smY, 0, ctx->ctrY)));
  }
  LaunchArgs x;
  x.p = ctx->p; x.st = ctx->st; x.ctr = ctx->ctrLL; x.n_pt_blocks = ctx->n_pt_blocks;
  x.apply_phi = 0; x.do_mu = 0; x.grid = dim3(ctx->n_pt_blocks);
  CK(launch(ctx, KK_XT, x));
  if (ctx->fusedPR) {
    // P, R of the first W update (later ones come from the IP kernel)
    Prob q = ctx->p;
    q.lam = ctx->lam;
    ctx->launches++;
    CK(launch_pr(ctx->maxm, q, ctx->PR, 0, ctx->st));
  }
  return FMNMF_OK;
}

// Copies the current state (W, H, G, Q) to the restart snapshot, or back from it.
fmnmf_status snapshot(fmnmf_ctx* ctx, bool restore) {
  const size_t F = ctx->F, T = ctx->T, M = ctx->M, N = ctx->N, K = ctx->K;
  struct { void* live; void* snap; size_t bytes; } c[4] = {
      {ctx->p.W, ctx->W0, N * K * F * 4}, {ctx->p.H, ctx->H0, N * K * T * 4},
      {ctx->p.G, ctx->G0, N * F * M * 4}, {ctx->p.Qx, ctx->Q0, F * M * M * sizeof(float4)}};
  for (auto& e : c)
    CK(cudaMemcpyAsync(restore ? e.live : e.snap, restore ? e.snap : e.live, e.bytes,
                       cudaMemcpyDeviceToDevice, ctx->st));
  if (ctx->free_model)
    CK(cudaMemcpyAsync(restore ? ctx->lam : ctx->lam0, restore ? ctx->lam0 : ctx->lam, N * F * T * 4,
                       cudaMemcpyDeviceToDevice, ctx->st));
  return FMNMF_OK;
}

fmnmf_status check_status(fmnmf_ctx* ctx) {
  unsigned st = 0;
  CK(cudaMemcpyAsync(&st, ctx->p.status, 4, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  // a wait that ran out leaves results undefined downstream (which may then look singular or
  // non-finite): it is the cause to report
  if (st & ST_TIMEOUT) return set_err(ctx, FMNMF_ETIMEOUT, "device wait timed out (status 0x%x)", st);
  if (st & ST_SINGULAR) return set_err(ctx, FMNMF_ESINGULAR, "singular IP system or diagonaliser (device status 0x%x)", st);
  if (st & ST_NONFINITE) return set_err(ctx, FMNMF_ENONFINITE, "non-finite value produced on the device (status 0x%x)", st);
  return FMNMF_OK;
}

void harvest(fmnmf_ctx* c, std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>>& ev, bool release) {
  for (auto& k : ev) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, k.second.first, k.second.second) == cudaSuccess) {
      c->ms[k.first] += ms;
      c->cnt[k.first] += 1;
    }
    if (release) { c->evpool.push_back(k.second.first); c->evpool.push_back(k.second.second); }
  }
  if (release) ev.clear();
}

// SplitMix64 (Steele, Lea & Flood 2014), counter form: output i of the stream seeded
// with s is mix(s + (i + 1) * 0x9E3779B97F4A7C15).
inline uint64_t sm64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// The first non-finite float of x[0..n) (atomicMin of its index; *first starts at all ones).
__global__ void k_check_finite(const float* __restrict__ x, size_t n, unsigned long long* first) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) atomicMin(first, (unsigned long long)i);
}

// Copies X into the context (host -> device or device -> device) and checks it on the
// device: the first non-finite float, if any, is reported as FMNMF_ENONFINITE (the copy has
// then replaced the context's mixture).  Synchronises.
fmnmf_status load_x(fmnmf_ctx* ctx, const void* X, int x_on_device) {
  const size_t nfl = (size_t)ctx->F * ctx->T * ctx->M * 2;
  if (!X) return set_err(ctx, FMNMF_EINVAL, "X is NULL");
  CK(cudaMemcpyAsync((void*)ctx->p.X, X, nfl * 4, x_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     ctx->st));
  // the per-CTA log-likelihood partials are scratch between launches: their first 8 bytes
  // hold the index
  unsigned long long* first = reinterpret_cast<unsigned long long*>(ctx->p.llpart);
  CK(cudaMemsetAsync(first, 0xFF, sizeof(unsigned long long), ctx->st));
  const unsigned blocks = (unsigned)std::min<size_t>((size_t)4 * std::max(1, ctx->sms), (nfl + 255) / 256);
  k_check_finite<<<blocks, 256, 0, ctx->st>>>((const float*)ctx->p.X, nfl, first);
  CK(cudaGetLastError());
  unsigned long long h = 0;
  CK(cudaMemcpyAsync(&h, first, sizeof h, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (h != ~0ULL) return set_err(ctx, FMNMF_ENONFINITE, "X has a non-finite value at float %llu", h);
  return FMNMF_OK;
}

fmnmf_status seed_state(fmnmf_ctx* ctx, uint64_t seed) {
  const int F = ctx->F, T = ctx->T, M = ctx->M, N = ctx->N, K = ctx->K;
  const size_t nw = (size_t)N * K * F, nh = (size_t)N * K * T;
  std::vector<float> W(nw), H(nh), G((size_t)N * F * M);
  std::vector<float4> Q((size_t)F * M * M);
  for (size_t i = 0; i < nw; ++i) W[i] = (float)(0.1 + (double)(sm64(seed, i) >> 11) * 0x1.0p-53);
  for (size_t i = 0; i < nh; ++i) H[i] = (float)(0.1 + (double)(sm64(seed, nw + i) >> 11) * 0x1.0p-53);
  for (int n = 0; n < N; ++n) {
    double sum = 0.0;
    for (int m = 0; m < M; ++m) sum += (m == n % M) ? 1.0 : 1e-2;
    for (int f = 0; f < F; ++f)
      for (int m = 0; m < M; ++m) G[((size_t)n * F + f) * M + m] = (float)(((m == n % M) ? 1.0 : 1e-2) / sum);
  }
  for (int f = 0; f < F; ++f)
    for (int i = 0; i < M; ++i)
      for (int j = 0; j < M; ++j) Q[((size_t)f * M + i) * M + j] = make_float4(i == j ? 1.f : 0.f, 0.f, 0.f, 0.f);
  CK(cudaMemcpyAsync(ctx->p.W, W.data(), nw * 4, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->p.H, H.data(), nh * 4, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->p.G, G.data(), G.size() * 4, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->p.Qx, Q.data(), Q.size() * sizeof(float4), cudaMemcpyHostToDevice, ctx->st));
  std::vector<float> L;
  if (ctx->free_model) {
    // lambda[n][f][t] = 0.1 + u_{(nF + f)T + t}
    const size_t nl = (size_t)N * F * T;
    L.resize(nl);
    for (size_t i = 0; i < nl; ++i) L[i] = (float)(0.1 + (double)(sm64(seed, i) >> 11) * 0x1.0p-53);
    CK(cudaMemcpyAsync(ctx->lam, L.data(), nl * 4, cudaMemcpyHostToDevice, ctx->st));
  }
  CK(cudaMemsetAsync(ctx->p.status, 0, 4, ctx->st));
  // the host vectors die at return: wait for the copies
  CK(cudaStreamSynchronize(ctx->st));
  return FMNMF_OK;
}

// Failure-detection tests only: FMNMF_TEST_WAIT_LIMIT (a count of tries) replaces the bound
// of the tensor-core kernels' consumer waits, and one of their waits then goes to an mbarrier
// nothing arrives at, so that their timeout path runs (the CTA leaves its loop, drains the
// copies and MMAs it issued with the full bound, reports ST_TIMEOUT and frees its TMEM).
// Read at context creation and at every fmnmf_iterate; unset (the normal case) it is 0.
unsigned test_wait_limit() {
  const char* wl = std::getenv("FMNMF_TEST_WAIT_LIMIT");
  return wl ? (unsigned)std::strtoul(wl, nullptr, 10) : 0u;
}

void clear_graphs(fmnmf_ctx* ctx);

// Picks up a changed test wait limit before a call launches kernels (graphs recaptured).
void sync_wait_limit(fmnmf_ctx* ctx) {
  const unsigned wl = test_wait_limit();
  if (wl == ctx->p.wait_limit) return;
  clear_graphs(ctx);
  ctx->p.wait_limit = wl;
  ctx->gpW.g.wait_limit = ctx->gpH.g.wait_limit = ctx->gpL.g.wait_limit = wl;
}

// Drops the captured graphs (their launch shapes changed).
void clear_graphs(fmnmf_ctx* ctx) {
  if (ctx->st) cudaStreamSynchronize(ctx->st);
  for (auto& kv : ctx->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    for (auto& e : kv.second.ev) { cudaEventDestroy(e.second.first); cudaEventDestroy(e.second.second); }
  }
  ctx->graphs.clear();
}

// An exact copy of everything an iteration changes (W, H, g~, Q and Q^-1 in both storage
// forms, log|det Q|^2, phi, x~, y~, the log-likelihood and, in the mixed form, lambda) for
// the tuner's trials; restoring it makes the context continue bit for bit as it would have.
struct SavedState {
  void* buf = nullptr;
  std::vector<std::pair<void*, size_t>> arrays;  // live array, bytes
  std::vector<size_t> off;
};
fmnmf_status save_state(fmnmf_ctx* ctx, SavedState& sv) {
  const size_t F = ctx->F, T = ctx->T, M = ctx->M, N = ctx->N, K = ctx->K;
  Prob& p = ctx->p;
  sv.arrays = {{p.W, N * K * F * 4}, {p.H, N * K * T * 4}, {p.G, N * F * M * 4},
               {p.Qx, F * M * M * sizeof(float4)}, {p.Qix, F * M * M * sizeof(float4)},
               {p.Qf, F * M * M * sizeof(float2)}, {p.Qinv, F * M * M * sizeof(float2)},
               {p.logdet, F * 8}, {p.phi, F * 4}, {p.xt, F * T * M * 4}, {p.yt, F * T * M * 4}, {p.ll, 8}};
  if (ctx->mixed || ctx->fused) sv.arrays.push_back({ctx->lam, N * F * T * 4});
  if (ctx->fusedPR) sv.arrays.push_back({ctx->PR, 2 * N * F * T * 4});  // P, R of the next W update
  size_t tot = 0;
  for (auto& a : sv.arrays) { sv.off.push_back(tot); tot += (a.second + 255) & ~(size_t)255; }
  cudaError_t e = cudaMallocAsync(&sv.buf, tot, ctx->st);
  if (e != cudaSuccess) return set_err(ctx, FMNMF_ENOMEM, "tuner state copy (%zu bytes): %s", tot, cudaGetErrorString(e));
  for (size_t i = 0; i < sv.arrays.size(); ++i)
    CK(cudaMemcpyAsync((char*)sv.buf + sv.off[i], sv.arrays[i].first, sv.arrays[i].second, cudaMemcpyDeviceToDevice,
                       ctx->st));
  return FMNMF_OK;
}
fmnmf_status restore_state(fmnmf_ctx* ctx, const SavedState& sv) {
  for (size_t i = 0; i < sv.arrays.size(); ++i)
    CK(cudaMemcpyAsync(sv.arrays[i].first, (char*)sv.buf + sv.off[i], sv.arrays[i].second, cudaMemcpyDeviceToDevice,
                       ctx->st));
  CK(cudaMemsetAsync(ctx->p.status, 0, 4, ctx->st));
  return FMNMF_OK;
}

void free_ctx(fmnmf_ctx* ctx) {
  if (!ctx) return;
  if (ctx->st) cudaStreamSynchronize(ctx->st);
  for (auto& kv : ctx->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    for (auto& e : kv.second.ev) { cudaEventDestroy(e.second.first); cudaEventDestroy(e.second.second); }
  }
  for (auto& e : ctx->pending) { cudaEventDestroy(e.second.first); cudaEventDestroy(e.second.second); }
  for (auto e : ctx->evpool) cudaEventDestroy(e);
  if (ctx->arena) {
    cudaFreeAsync(ctx->arena, ctx->st);
    cudaStreamSynchronize(ctx->st);
  }
  if (ctx->own_stream && ctx->st) cudaStreamDestroy(ctx->st);
  delete ctx;
}

}  // namespace

namespace fm {
void set_thread_error(const char* msg) { g_thread_err = msg; }
}  // namespace fm

// =====================================================================================
// C ABI
// =====================================================================================
extern "C" {

fmnmf_status fmnmf_default_opts(fmnmf_opts* opts) {
  if (!opts) return set_err(nullptr, FMNMF_EINVAL, "opts is NULL");
  opts->precision = FMNMF_PREC_FP32;
  opts->update_mask = FMNMF_UPDATE_ALL;
  opts->normalise = 1;
  opts->stream = nullptr;
  opts->hbm_budget = 0;
  opts->schedule = FMNMF_SCHED_AUTO;
  opts->source_model = FMNMF_SOURCE_NMF;
  return FMNMF_OK;
}

fmnmf_status fmnmf_init(fmnmf_ctx** out, const void* X, int x_on_device, int F, int T, int M, int N,
                        int K, uint64_t seed, const fmnmf_opts* opts) {
  if (!out) return set_err(nullptr, FMNMF_EINVAL, "out is NULL");
  *out = nullptr;
  if (F < 1 || T < 1 || M < 1 || M > kMaxM || N < 1 || K < 1)
    return set_err(nullptr, FMNMF_EINVAL, "bad shape F=%d T=%d M=%d N=%d K=%d (need F,T,N,K >= 1, 1 <= M <= 8)", F, T, M, N, K);
  if ((double)F * T * M > 2.0e9) return set_err(nullptr, FMNMF_EINVAL, "F*T*M too large (> 2e9)");
  if (!X) return set_err(nullptr, FMNMF_EINVAL, "X is NULL");
  if (opts && (opts->precision < FMNMF_PREC_FP32 || opts->precision > FMNMF_PREC_TF32))
    return set_err(nullptr, FMNMF_EINVAL, "unknown precision %d", opts->precision);
  if (opts && (opts->schedule < FMNMF_SCHED_AUTO || opts->schedule > FMNMF_SCHED_FUSED))
    return set_err(nullptr, FMNMF_EINVAL, "unknown schedule %d", opts->schedule);
  if (opts && (opts->source_model < FMNMF_SOURCE_NMF || opts->source_model > FMNMF_SOURCE_FREE))
    return set_err(nullptr, FMNMF_EINVAL, "unknown source model %d", opts->source_model);
  if (opts && opts->source_model == FMNMF_SOURCE_FREE && opts->precision != FMNMF_PREC_FP32)
    return set_err(nullptr, FMNMF_EINVAL, "the unconstrained source model runs in the FP32 form only");
  fmnmf_ctx* ctx = new fmnmf_ctx();
  ctx->F = F; ctx->T = T; ctx->M = M; ctx->N = N; ctx->K = K; ctx->maxm = bucket(M);
  if (opts) ctx->opts = *opts; else fmnmf_default_opts(&ctx->opts);
  ctx->mixed = ctx->opts.precision != FMNMF_PREC_FP32;
  ctx->tf32 = ctx->opts.precision == FMNMF_PREC_TF32;
  ctx->free_model = ctx->opts.source_model == FMNMF_SOURCE_FREE;
  ctx->p.wait_limit = test_wait_limit();
  if (ctx->opts.update_mask & ~(unsigned)FMNMF_UPDATE_ALL) {
    const unsigned bad = ctx->opts.update_mask;
    delete ctx;
    return set_err(nullptr, FMNMF_EINVAL, "bad update_mask 0x%x", bad);
  }
  fmnmf_status s;
  if (ctx->opts.stream) {
    ctx->st = (cudaStream_t)ctx->opts.stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&ctx->st, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete ctx; return set_err(nullptr, FMNMF_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e)); }
    ctx->own_stream = true;
  }
  if ((s = plan(ctx)) != FMNMF_OK || (s = allocate(ctx)) != FMNMF_OK || (s = load_x(ctx, X, x_on_device)) != FMNMF_OK ||
      (s = seed_state(ctx, seed)) != FMNMF_OK || (s = snapshot(ctx, false)) != FMNMF_OK ||
      (s = refresh_state(ctx)) != FMNMF_OK || (s = check_status(ctx)) != FMNMF_OK) {
    g_thread_err = ctx->err;
    free_ctx(ctx);
    return s;
  }
  *out = ctx;
  return FMNMF_OK;
}

fmnmf_status fmnmf_footprint(int F, int T, int M, int N, int K, const fmnmf_opts* opts, size_t* bytes) {
  if (!bytes) return set_err(nullptr, FMNMF_EINVAL, "bytes is NULL");
  if (F < 1 || T < 1 || M < 1 || M > kMaxM || N < 1 || K < 1)
    return set_err(nullptr, FMNMF_EINVAL, "bad shape F=%d T=%d M=%d N=%d K=%d", F, T, M, N, K);
  fmnmf_ctx tmp;
  tmp.F = F; tmp.T = T; tmp.M = M; tmp.N = N; tmp.K = K; tmp.maxm = bucket(M);
  if (opts) tmp.opts = *opts; else fmnmf_default_opts(&tmp.opts);
  tmp.mixed = tmp.opts.precision != FMNMF_PREC_FP32;
  tmp.tf32 = tmp.opts.precision == FMNMF_PREC_TF32;
  tmp.free_model = tmp.opts.source_model == FMNMF_SOURCE_FREE;
  fmnmf_status s = plan(&tmp);
  if (s == FMNMF_OK) s = allocate(&tmp, true);
  if (s != FMNMF_OK) { g_thread_err = tmp.err; return s; }
  // the Wiener filter's output buffer when the result goes to the host
  *bytes = tmp.arena_bytes + (size_t)N * F * T * M * sizeof(float2);
  return FMNMF_OK;
}

fmnmf_status fmnmf_reset(fmnmf_ctx* ctx, const void* X, int x_on_device, uint64_t seed) {
  if (!ctx) return set_err(nullptr, FMNMF_EINVAL, "ctx is NULL");
  fmnmf_status s;
  if ((s = load_x(ctx, X, x_on_device)) != FMNMF_OK) return s;
  if ((s = seed_state(ctx, seed)) != FMNMF_OK) return s;
  if ((s = snapshot(ctx, false)) != FMNMF_OK) return s;
  if ((s = refresh_state(ctx)) != FMNMF_OK) return s;
  return FMNMF_OK;
}

fmnmf_status fmnmf_restart(fmnmf_ctx* ctx) {
  if (!ctx) return set_err(nullptr, FMNMF_EINVAL, "ctx is NULL");
  fmnmf_status s;
  if ((s = snapshot(ctx, true)) != FMNMF_OK) return s;
  CK(cudaMemsetAsync(ctx->p.status, 0, 4, ctx->st));
  return refresh_state(ctx);
}

fmnmf_status fmnmf_iterate(fmnmf_ctx* ctx, int n_iter) {
  if (!ctx) return set_err(nullptr, FMNMF_EINVAL, "ctx is NULL");
  if (n_iter < 0) return set_err(ctx, FMNMF_EINVAL, "n_iter < 0");
  sync_wait_limit(ctx);
  while (n_iter > 0) {
    const int chunk = std::min(n_iter, kMaxChunk);
    auto key = std::make_pair(chunk, ctx->timing);
    auto it = ctx->graphs.find(key);
    if (it == ctx->graphs.end()) {
      GraphEntry ge;
      cudaGraph_t g = nullptr;
      CK(cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal));
      Recorder rec{ctx, ctx->timing ? &ge.ev : nullptr};
      const long long before = ctx->launches;
      cudaError_t e = enqueue_chunk(ctx, rec, chunk);
      ge.launches = (int)(ctx->launches - before);
      ctx->launches = before;
      cudaError_t e2 = cudaStreamEndCapture(ctx->st, &g);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return set_err(ctx, FMNMF_ECUDA, "graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
      }
      CK(cudaGraphInstantiate(&ge.exec, g, 0));
      cudaGraphDestroy(g);
      it = ctx->graphs.emplace(key, std::move(ge)).first;
    }
    GraphEntry& ge = it->second;
    if (ctx->timing && ge.unharvested) {
      // the events of this graph still hold its previous launch: wait for that launch
      // only (work queued after it keeps the device busy) and accumulate it
      CK(cudaEventSynchronize(ge.ev.back().second.second));
      harvest(ctx, ge.ev, false);
      ge.unharvested = false;
    }
    CK(cudaGraphLaunch(ge.exec, ctx->st));
    ctx->launches += ge.launches;
    if (ctx->timing) ge.unharvested = true;
    n_iter -= chunk;
  }
  return FMNMF_OK;
}

fmnmf_status fmnmf_sync(fmnmf_ctx* ctx) {
  if (!ctx) return set_err(nullptr, FMNMF_EINVAL, "ctx is NULL");
  return check_status(ctx);
}

fmnmf_status fmnmf_query(fmnmf_ctx* ctx) {
  if (!ctx) return set_err(nullptr, FMNMF_EINVAL, "ctx is NULL");
  const cudaError_t e = cudaStreamQuery(ctx->st);
  if (e == cudaErrorNotReady) return FMNMF_EBUSY;
  if (e != cudaSuccess) return set_err(ctx, FMNMF_ECUDA, "cudaStreamQuery: %s", cudaGetErrorString(e));
  return check_status(ctx);  // the stream is idle: this does not wait
}

fmnmf_status fmnmf_loglik(fmnmf_ctx* ctx, double* ll) {
  if (!ctx || !ll) return set_err(ctx, FMNMF_EINVAL, "NULL argument");
  fmnmf_status s = check_status(ctx);
  if (s != FMNMF_OK) return s;
  CK(cudaMemcpyAsync(ll, ctx->p.ll, 8, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return FMNMF_OK;
}

fmnmf_status fmnmf_separate(fmnmf_ctx* ctx, void* out, int out_on_device) {
  if (!ctx || !out) return set_err(ctx, FMNMF_EINVAL, "NULL argument");
  const size_t bytes = (size_t)ctx->N * ctx->F * ctx->T * ctx->M * sizeof(float2);
  float2* dst = (float2*)out;
  float2* tmp = nullptr;
  if (!out_on_device) {
    cudaError_t e = cudaMallocAsync((void**)&tmp, bytes, ctx->st);
    if (e != cudaSuccess) return set_err(ctx, FMNMF_ENOMEM, "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
    dst = tmp;
  }
  // Q_f^-1 is kept current by the IP update (and by the preparation of a set state)
  sync_wait_limit(ctx);
  Recorder rec{ctx, ctx->timing ? &ctx->pending : nullptr};
  LaunchArgs a;
  a.p = ctx->p; a.g = ctx->gS; a.smem = ctx->smS; a.st = ctx->st; a.out = dst;
  if (ctx->mixed) {
    // lambda of the current W and H (the normalisation rescaled W after the last GEMM),
    // with split-BF16 operands (about 16 significant bits) in either mixed form: the images
    // scale with lambda directly
    cudaError_t el = rec.run_fn(KK_GL, [&] {
      ctx->launches++;
      return launch_gemm(ctx->gpL.g, false, ctx->gpL.nt, ctx->gpL.grid, ctx->st);
    });
    if (el != cudaSuccess) {
      if (tmp) cudaFreeAsync(tmp, ctx->st);
      return set_err(ctx, FMNMF_ECUDA, "lambda GEMM launch: %s", cudaGetErrorString(el));
    }
    a.p.lam = ctx->lam;
  } else if (ctx->free_model) {
    a.p.lam = ctx->lam;  // the lambda state (nu already applied)
  }
  a.grid = dim3(ctx->gS.n_own_tiles, ctx->gS.S);
  cudaError_t e = rec.run(KK_SEP, a);
  if (e != cudaSuccess) {
    if (tmp) cudaFreeAsync(tmp, ctx->st);
    return set_err(ctx, FMNMF_ECUDA, "separate launch: %s", cudaGetErrorString(e));
  }
  if (!out_on_device) {
    CK(cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaFreeAsync(tmp, ctx->st));
    return check_status(ctx);
  }
  return FMNMF_OK;
}

fmnmf_status fmnmf_get_state(fmnmf_ctx* ctx, float* W, float* H, float* G, void* Q) {
  if (!ctx) return set_err(nullptr, FMNMF_EINVAL, "ctx is NULL");
  if (ctx->free_model && (W || H))
    return set_err(ctx, FMNMF_EINVAL, "the unconstrained source model has no W, H (use fmnmf_get_lambda)");
  CK(cudaStreamSynchronize(ctx->st));
  const size_t F = ctx->F, T = ctx->T, M = ctx->M, N = ctx->N, K = ctx->K;
  if (W) CK(cudaMemcpyAsync(W, ctx->p.W, N * K * F * 4, cudaMemcpyDeviceToHost, ctx->st));
  if (H) CK(cudaMemcpyAsync(H, ctx->p.H, N * K * T * 4, cudaMemcpyDeviceToHost, ctx->st));
  if (G) CK(cudaMemcpyAsync(G, ctx->p.G, N * F * M * 4, cudaMemcpyDeviceToHost, ctx->st));
  if (Q) CK(cudaMemcpyAsync(Q, ctx->p.Qf, F * M * M * sizeof(float2), cudaMemcpyDeviceToHost, ctx->st));
  return check_status(ctx);
}

// Validates g~ and Q from the host and converts Q to the float-float storage form.
static fmnmf_status check_gq(fmnmf_ctx* ctx, const float* G, const void* Q, std::vector<float4>& Qx) {
  const size_t F = ctx->F, M = ctx->M, N = ctx->N;
  for (size_t i = 0; i < N * F * M; ++i)
    if (!(G[i] >= 0.f) || !std::isfinite(G[i])) return set_err(ctx, FMNMF_EINVAL, "g~ must be finite and nonnegative");
  const float* q = (const float*)Q;
  Qx.resize(F * M * M);
  for (size_t i = 0; i < F * M * M; ++i) {
    if (!std::isfinite(q[2 * i]) || !std::isfinite(q[2 * i + 1])) return set_err(ctx, FMNMF_EINVAL, "Q must be finite");
    Qx[i] = make_float4(q[2 * i], 0.f, q[2 * i + 1], 0.f);
  }
  return FMNMF_OK;
}

fmnmf_status fmnmf_get_lambda(fmnmf_ctx* ctx, float* lam, float* G, void* Q) {
  if (!ctx || !lam) return set_err(ctx, FMNMF_EINVAL, "get_lambda: NULL argument");
  if (!ctx->free_model) return set_err(ctx, FMNMF_EINVAL, "get_lambda: the context has the NMF source model");
  CK(cudaStreamSynchronize(ctx->st));
  const size_t F = ctx->F, T = ctx->T, M = ctx->M, N = ctx->N;
  CK(cudaMemcpyAsync(lam, ctx->lam, N * F * T * 4, cudaMemcpyDeviceToHost, ctx->st));
  if (G) CK(cudaMemcpyAsync(G, ctx->p.G, N * F * M * 4, cudaMemcpyDeviceToHost, ctx->st));
  if (Q) CK(cudaMemcpyAsync(Q, ctx->p.Qf, F * M * M * sizeof(float2), cudaMemcpyDeviceToHost, ctx->st));
  return check_status(ctx);
}

fmnmf_status fmnmf_set_lambda(fmnmf_ctx* ctx, const float* lam, const float* G, const void* Q) {
  if (!ctx) return set_err(nullptr, FMNMF_EINVAL, "ctx is NULL");
  if (!lam || !G || !Q) return set_err(ctx, FMNMF_EINVAL, "set_lambda needs lambda, g~ and Q");
  if (!ctx->free_model) return set_err(ctx, FMNMF_EINVAL, "set_lambda: the context has the NMF source model");
  const size_t F = ctx->F, T = ctx->T, M = ctx->M, N = ctx->N;
  for (size_t i = 0; i < N * F * T; ++i)
    if (!(lam[i] >= 0.f) || !std::isfinite(lam[i])) return set_err(ctx, FMNMF_EINVAL, "lambda must be finite and nonnegative");
  std::vector<float4> Qx;
  fmnmf_status s = check_gq(ctx, G, Q, Qx);
  if (s != FMNMF_OK) return s;
  CK(cudaStreamSynchronize(ctx->st));
  CK(cudaMemcpyAsync(ctx->lam, lam, N * F * T * 4, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->p.G, G, N * F * M * 4, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->p.Qx, Qx.data(), Qx.size() * sizeof(float4), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemsetAsync(ctx->p.status, 0, 4, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));  // the host vector Qx goes out of scope
  if ((s = snapshot(ctx, false)) != FMNMF_OK) return s;
  if ((s = refresh_state(ctx)) != FMNMF_OK) return s;
  return check_status(ctx);
}

fmnmf_status fmnmf_set_state(fmnmf_ctx* ctx, const float* W, const float* H, const float* G, const void* Q) {
  if (!ctx) return set_err(nullptr, FMNMF_EINVAL, "ctx is NULL");
  if (ctx->free_model) return set_err(ctx, FMNMF_EINVAL, "the unconstrained source model has no W, H (use fmnmf_set_lambda)");
  if (!W || !H || !G || !Q) return set_err(ctx, FMNMF_EINVAL, "set_state needs W, H, G and Q");
  const size_t F = ctx->F, T = ctx->T, M = ctx->M, N = ctx->N, K = ctx->K;
  auto nonneg = [](const float* a, size_t n) {
    for (size_t i = 0; i < n; ++i) if (!(a[i] >= 0.f) || !std::isfinite(a[i])) return false;
    return true;
  };
  if (!nonneg(W, N * K * F) || !nonneg(H, N * K * T) || !nonneg(G, N * F * M))
    return set_err(ctx, FMNMF_EINVAL, "W, H and G must be finite and nonnegative");
  const float* q = (const float*)Q;
  std::vector<float4> Qx(F * M * M);
  for (size_t i = 0; i < F * M * M; ++i) {
    if (!std::isfinite(q[2 * i]) || !std::isfinite(q[2 * i + 1])) return set_err(ctx, FMNMF_EINVAL, "Q must be finite");
    Qx[i] = make_float4(q[2 * i], 0.f, q[2 * i + 1], 0.f);
  }
  CK(cudaStreamSynchronize(ctx->st));
  CK(cudaMemcpyAsync(ctx->p.W, W, N * K * F * 4, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->p.H, H, N * K * T * 4, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->p.G, G, N * F * M * 4, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->p.Qx, Qx.data(), Qx.size() * sizeof(float4), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemsetAsync(ctx->p.status, 0, 4, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));  // the host vector Qx goes out of scope
  fmnmf_status s = snapshot(ctx, false);
  if (s != FMNMF_OK) return s;
  s = refresh_state(ctx);
  if (s != FMNMF_OK) return s;
  return check_status(ctx);
}

// Spectral initialisation (Sec. IV-A): g~ and Q from the eigendecomposition of the average
// observed SCM (one float64 Jacobi solve per bin on the device), then the nu normalisation
// with W (or lambda) scaled to match; H is kept.  Replaces the state like fmnmf_set_state.
fmnmf_status fmnmf_init_spectral(fmnmf_ctx* ctx) {
  if (!ctx) return set_err(nullptr, FMNMF_EINVAL, "ctx is NULL");
  CK(cudaStreamSynchronize(ctx->st));
  CK(cudaMemsetAsync(ctx->p.status, 0, 4, ctx->st));
  ctx->launches++;
  CK(launch_spec_init(ctx->p, ctx->free_model ? ctx->lam : nullptr, ctx->st));
  fmnmf_status s = check_status(ctx);
  if (s != FMNMF_OK) return s;
  if ((s = snapshot(ctx, false)) != FMNMF_OK) return s;
  if ((s = refresh_state(ctx)) != FMNMF_OK) return s;
  return check_status(ctx);
}

fmnmf_status fmnmf_shape(const fmnmf_ctx* ctx, int* F, int* T, int* M, int* N, int* K) {
  if (!ctx) return set_err(nullptr, FMNMF_EINVAL, "ctx is NULL");
  if (F) *F = ctx->F;
  if (T) *T = ctx->T;
  if (M) *M = ctx->M;
  if (N) *N = ctx->N;
  if (K) *K = ctx->K;
  return FMNMF_OK;
}

fmnmf_status fmnmf_destroy(fmnmf_ctx* ctx) {
  free_ctx(ctx);
  return FMNMF_OK;
}

const char* fmnmf_last_error(const fmnmf_ctx* ctx) { return ctx ? ctx->err.c_str() : g_thread_err.c_str(); }

fmnmf_status fmnmf_set_timing(fmnmf_ctx* ctx, int kinds) {
  if (!ctx) return set_err(nullptr, FMNMF_EINVAL, "ctx is NULL");
  ctx->timing = (unsigned)kinds & ((1u << KK_COUNT) - 1u);
  return FMNMF_OK;
}

fmnmf_status fmnmf_kernel_times(fmnmf_ctx* ctx, double* ms, long long* launches, int* n) {
  if (!ctx || !n) return set_err(ctx, FMNMF_EINVAL, "NULL argument");
  CK(cudaStreamSynchronize(ctx->st));
  harvest(ctx, ctx->pending, true);
  for (auto& kv : ctx->graphs)
    if (kv.second.unharvested) { harvest(ctx, kv.second.ev, false); kv.second.unharvested = false; }
  const int cap = *n;
  for (int i = 0; i < KK_COUNT && i < cap; ++i) {
    if (ms) ms[i] = ctx->ms[i];
    if (launches) launches[i] = ctx->cnt[i];
    ctx->ms[i] = 0.0;
    ctx->cnt[i] = 0;
  }
  *n = KK_COUNT;
  return FMNMF_OK;
}

const char* fmnmf_kernel_name(int i) { return (i >= 0 && i < KK_COUNT) ? kKindNames[i] : ""; }

long long fmnmf_launch_count(const fmnmf_ctx* ctx) { return ctx ? ctx->launches : 0; }

// ---- batches ---------------------------------------------------------------------------
// One timed trial of the current launch shapes: n_iter iterations from the saved state (the
// graph captured and run once untimed, then timed), in milliseconds; +inf if it failed.
static double tune_trial(fmnmf_ctx* ctx, const SavedState& sv, int n_iter, cudaEvent_t e0, cudaEvent_t e1) {
  clear_graphs(ctx);
  if (restore_state(ctx, sv) != FMNMF_OK || fmnmf_iterate(ctx, n_iter) != FMNMF_OK) return INFINITY;
  if (restore_state(ctx, sv) != FMNMF_OK) return INFINITY;
  if (cudaEventRecord(e0, ctx->st) != cudaSuccess || fmnmf_iterate(ctx, n_iter) != FMNMF_OK ||
      cudaEventRecord(e1, ctx->st) != cudaSuccess || check_status(ctx) != FMNMF_OK)
    return INFINITY;
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return INFINITY;
  return ms;
}

// Split-count scales the tuner tries.  The planner aims at two or more waves (HBM-bound
// mixtures); the in-between scales reach one-wave shapes of short mixtures, where a CTA
// that pipelines a few stages beats two waves of one-stage CTAs.
static const float kTuneScales[] = {1.f, 0.75f, 0.5f, 0.375f, 0.25f, 0.1875f, 0.125f};

fmnmf_status fmnmf_autotune(fmnmf_ctx* ctx, int n_iter, double* speedup) {
  if (!ctx || n_iter < 1) return set_err(ctx, FMNMF_EINVAL, "autotune: bad arguments");
  SavedState sv;
  fmnmf_status s = save_state(ctx, sv);
  if (s != FMNMF_OK) return s;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // the fused schedule's one tunable launch shape is the H kernel's frame tile (entry TU_H)
  std::vector<int> tun;
  if (ctx->fused) tun = {};  // no tunable launch shape (bins per CTA and splits are fixed)
  else if (ctx->mixed) tun = {TU_SCM, TU_GTC, TU_GEMM_W, TU_GEMM_H};
  else tun = {TU_W, TU_H, TU_G, TU_Y};
  const double t0 = tune_trial(ctx, sv, n_iter, e0, e1);
  double best = t0;
  // coordinate descent over the split scales, two passes
  for (int pass = 0; pass < 2; ++pass)
    for (int t : tun) {
      if (t == TU_GTC && ctx->gtcNP == 0) continue;
      const float keep = ctx->tscale[t];
      float pick = keep;
      for (float sc : kTuneScales) {
        if (sc == keep) continue;
        ctx->tscale[t] = sc;
        apply_shapes(ctx);
        const double ms = tune_trial(ctx, sv, n_iter, e0, e1);
        if (ms < 0.98 * best) { best = ms; pick = sc; }
      }
      ctx->tscale[t] = pick;
      apply_shapes(ctx);
    }
  clear_graphs(ctx);
  s = restore_state(ctx, sv);
  cudaFreeAsync(sv.buf, ctx->st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != FMNMF_OK) return s;
  if (speedup) *speedup = (std::isfinite(t0) && std::isfinite(best) && best > 0) ? t0 / best : 1.0;
  return check_status(ctx);
}

fmnmf_status fmnmf_get_tuning(const fmnmf_ctx* ctx, float* scales) {
  if (!ctx || !scales) return set_err(nullptr, FMNMF_EINVAL, "get_tuning: NULL argument");
  for (int t = 0; t < TU_COUNT; ++t) scales[t] = ctx->tscale[t];
  return FMNMF_OK;
}

fmnmf_status fmnmf_set_tuning(fmnmf_ctx* ctx, const float* scales) {
  if (!ctx || !scales) return set_err(ctx, FMNMF_EINVAL, "set_tuning: NULL argument");
  for (int t = 0; t < TU_COUNT; ++t)
    if (!(scales[t] > 0.f && scales[t] <= 1.f)) return set_err(ctx, FMNMF_EINVAL, "set_tuning: scale %d not in (0, 1]", t);
  for (int t = 0; t < TU_COUNT; ++t) ctx->tscale[t] = scales[t];
  apply_shapes(ctx);
  clear_graphs(ctx);
  return FMNMF_OK;
}

fmnmf_status fmnmf_batch_create(fmnmf_ctx* const* ctxs, int n, fmnmf_batch** out) {
  if (!out || !ctxs || n < 1) return set_err(nullptr, FMNMF_EINVAL, "batch_create: bad arguments");
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return set_err(nullptr, FMNMF_EINVAL, "batch_create: context %d is NULL", i);
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i] || ctxs[j]->st == ctxs[i]->st)
        return set_err(nullptr, FMNMF_EINVAL, "batch_create: contexts %d and %d share a stream", j, i);
  }
  fmnmf_batch* b = new fmnmf_batch();
  b->ctxs.assign(ctxs, ctxs + n);
  cudaError_t e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
  if (e != cudaSuccess) { delete b; return set_err(nullptr, FMNMF_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e)); }
  *out = b;
  return FMNMF_OK;
}

fmnmf_status fmnmf_batch_iterate(fmnmf_batch* b, int n_iter) {
  if (!b || n_iter < 0) return set_err(nullptr, FMNMF_EINVAL, "batch_iterate: bad arguments");
  fmnmf_ctx* ctx = nullptr;  // for CK
  while (n_iter > 0) {
    const int chunk = std::min(n_iter, kMaxChunk);
    auto it = b->graphs.find(chunk);
    if (it == b->graphs.end()) {
      // capture: fork every context stream off the origin stream, enqueue its iterations,
      // join back; the result is one graph whose branches run concurrently
      const int n = (int)b->ctxs.size();
      while ((int)b->events.size() < n + 1) {
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        b->events.push_back(ev);
      }
      cudaGraph_t g = nullptr;
      CK(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = cudaEventRecord(b->events[n], b->st);
      long long launches = 0;
      for (int i = 0; i < n && e == cudaSuccess; ++i) {
        fmnmf_ctx* c = b->ctxs[i];
        if ((e = cudaStreamWaitEvent(c->st, b->events[n], 0)) != cudaSuccess) break;
        Recorder rec{c, nullptr};
        const long long before = c->launches;
        e = enqueue_chunk(c, rec, chunk);
        launches += c->launches - before;
        c->launches = before;
        if (e == cudaSuccess) e = cudaEventRecord(b->events[i], c->st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->st, b->events[i], 0);
      }
      cudaError_t e2 = cudaStreamEndCapture(b->st, &g);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        b->err = std::string("batch graph capture failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2);
        return set_err(nullptr, FMNMF_ECUDA, "%s", b->err.c_str());
      }
      cudaGraphExec_t ex = nullptr;
      CK(cudaGraphInstantiate(&ex, g, 0));
      cudaGraphDestroy(g);
      it = b->graphs.emplace(chunk, ex).first;
      b->graph_launches[chunk] = launches;
    }
    // the origin stream must follow the work already queued on every member stream
    for (size_t i = 0; i < b->ctxs.size(); ++i) {
      CK(cudaEventRecord(b->events[i], b->ctxs[i]->st));
      CK(cudaStreamWaitEvent(b->st, b->events[i], 0));
    }
    CK(cudaGraphLaunch(it->second, b->st));
    // and every member stream must follow the graph before its own next work
    CK(cudaEventRecord(b->events[b->ctxs.size()], b->st));
    for (auto* c : b->ctxs) {
      CK(cudaStreamWaitEvent(c->st, b->events[b->ctxs.size()], 0));
    }
    // launch accounting: spread over the member contexts in proportion
    const long long per = b->graph_launches[chunk] / (long long)b->ctxs.size();
    for (auto* c : b->ctxs) c->launches += per;
    n_iter -= chunk;
  }
  return FMNMF_OK;
}

// The batch tuner: the members' split counts scaled together (one scale for every tunable
// launch of every member); each candidate timed on the whole batch, from saved states.
fmnmf_status fmnmf_batch_autotune(fmnmf_batch* b, int n_iter, double* speedup) {
  if (!b || n_iter < 1) return set_err(nullptr, FMNMF_EINVAL, "batch_autotune: bad arguments");
  fmnmf_ctx* ctx = nullptr;  // for CK
  const size_t n = b->ctxs.size();
  std::vector<SavedState> sv(n);
  for (size_t i = 0; i < n; ++i) {
    fmnmf_status s = save_state(b->ctxs[i], sv[i]);
    if (s != FMNMF_OK) {
      for (size_t j = 0; j < i; ++j) cudaFreeAsync(sv[j].buf, b->ctxs[j]->st);
      return s;
    }
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  auto drop_graphs = [&] {
    if (b->st) cudaStreamSynchronize(b->st);
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    b->graph_launches.clear();
  };
  auto restore_all = [&] {
    for (size_t i = 0; i < n; ++i)
      if (restore_state(b->ctxs[i], sv[i]) != FMNMF_OK) return false;
    for (auto* c : b->ctxs)
      if (cudaStreamSynchronize(c->st) != cudaSuccess) return false;
    return true;
  };
  auto trial = [&]() -> double {
    drop_graphs();
    if (!restore_all() || fmnmf_batch_iterate(b, n_iter) != FMNMF_OK) return INFINITY;
    if (!restore_all()) return INFINITY;
    if (cudaEventRecord(e0, b->st) != cudaSuccess || fmnmf_batch_iterate(b, n_iter) != FMNMF_OK ||
        cudaEventRecord(e1, b->st) != cudaSuccess || fmnmf_batch_sync(b) != FMNMF_OK)
      return INFINITY;
    float ms = 0.f;
    return cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess ? (double)ms : INFINITY;
  };
  auto set_all = [&](float sc) {
    for (auto* c : b->ctxs) {
      for (int t = 0; t < TU_COUNT; ++t) c->tscale[t] = sc;
      apply_shapes(c);
      clear_graphs(c);
    }
  };
  set_all(1.f);
  const double t0 = trial();
  double best = t0;
  float pick = 1.f;
  for (float sc : kTuneScales) {
    if (sc == 1.f) continue;
    set_all(sc);
    const double ms = trial();
    if (ms < 0.98 * best) { best = ms; pick = sc; }
  }
  set_all(pick);
  drop_graphs();
  const bool ok = restore_all();
  for (size_t i = 0; i < n; ++i) cudaFreeAsync(sv[i].buf, b->ctxs[i]->st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) return set_err(nullptr, FMNMF_ECUDA, "batch_autotune: restoring a member's state failed");
  if (speedup) *speedup = (std::isfinite(t0) && std::isfinite(best) && best > 0) ? t0 / best : 1.0;
  return fmnmf_batch_sync(b);
}

fmnmf_status fmnmf_batch_sync(fmnmf_batch* b) {
  if (!b) return set_err(nullptr, FMNMF_EINVAL, "batch is NULL");
  fmnmf_status worst = FMNMF_OK;
  for (auto* c : b->ctxs) {
    fmnmf_status s = check_status(c);
    if (s != FMNMF_OK && worst == FMNMF_OK) {
      worst = s;
      set_err(nullptr, s, "%s", c->err.c_str());
    }
  }
  return worst;
}

fmnmf_status fmnmf_batch_destroy(fmnmf_batch* b) {
  if (!b) return FMNMF_OK;
  if (b->st) cudaStreamSynchronize(b->st);
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  for (auto ev : b->events) cudaEventDestroy(ev);
  if (b->st) cudaStreamDestroy(b->st);
  delete b;
  return FMNMF_OK;
}

}  // extern "C"

// ===========================================================================================
// FastMNMF-DP (Sec. III-B-3, Sec. III-C-3): the deep-prior speech source (source 0) and NMF
// noise sources around a context of the unconstrained source model, whose lambda, g~, Q, x~
// and per-bin kernel (g~, V_fm + IP, normalisation, x~, terms of Eq. 17) it shares.
// ===========================================================================================
struct fmnmf_dp {
  fmnmf_ctx* ctx = nullptr;
  fmnmf_dp_opts o{};
  int F = 0, T = 0, M = 0, N = 0, K = 0;
  void* buf = nullptr;  // u, v, Z, R, noise W and H, decoder, nu, draws, log gamma, counter
  float *u = nullptr, *v = nullptr, *Z = nullptr, *R = nullptr, *Wn = nullptr, *Hn = nullptr;
  float *W1 = nullptr, *b1 = nullptr, *W2 = nullptr, *b2 = nullptr, *nu = nullptr;
  float *xi = nullptr, *logu = nullptr, *lg = nullptr;
  unsigned long long* acc = nullptr;
  int draw_iters = 0;  // iterations of host draws the device buffers hold
  DpMhPlan mh;  // launch shape of the Metropolis kernel
  bool have_decoder = false, have_state = false;
};

namespace {

constexpr int kDpDrawIters = 4;  // host draws are copied in chunks of this many iterations

DpArgs dp_args(fmnmf_dp* d) {
  DpArgs a;
  a.p = d->ctx->p;
  a.lam = d->ctx->lam;
  a.u = d->u; a.v = d->v; a.Z = d->Z; a.R = d->R; a.Wn = d->Wn; a.Hn = d->Hn;
  a.W1 = d->W1; a.b1 = d->b1; a.W2 = d->W2; a.b2 = d->b2;
  a.D = d->o.D; a.Hd = d->o.Hd; a.K = d->K;
  a.S = d->o.n_proposals;
  a.sqrt_eps = (float)std::sqrt((double)d->o.eps);
  a.n_acc = d->acc;
  a.nu = d->nu;
  a.maxm = d->ctx->maxm;
  a.tb = d->mh.TB;
  return a;
}

// One iteration: Z (S proposals per frame), u, v, the noise W, H, then the per-bin kernel
// (g~, Q, phi / nu normalisation with nu exported, x~, terms of Eq. 17), then nu / mu into
// u, v, W, H; with `last`, the sum of Eq. 17.
cudaError_t enqueue_dp_iteration(fmnmf_dp* d, const float* xi, const float* logu, bool last) {
  fmnmf_ctx* c = d->ctx;
  DpArgs a = dp_args(d);
  a.xi = xi;
  a.logu = logu;
  const bool norm = d->o.normalise != 0;
  cudaError_t e;
  if (a.S > 0) {
    c->launches++;
    if ((e = dp_launch_mh(a, d->mh, c->st)) != cudaSuccess) return e;
  }
  c->launches += 2;
  if ((e = dp_launch_fsweep(a, 0, c->st)) != cudaSuccess) return e;
  if ((e = dp_launch_tsweep(a, 0, c->st)) != cudaSuccess) return e;
  if (d->N > 1) {
    c->launches += 2;
    if ((e = dp_launch_fsweep(a, 1, c->st)) != cudaSuccess) return e;
    if ((e = dp_launch_tsweep(a, 1, c->st)) != cudaSuccess) return e;
  }
  LaunchArgs b;
  b.p = c->p;
  b.p.nu_out = d->nu;
  b.st = c->st;
  b.grid = dim3(c->F);
  b.smem = c->binSm;
  b.flags = FU_G | FU_Q | FU_FREE | (norm ? (FU_NORM | FU_LAMWB) : 0);
  b.lam = c->lam;
  b.pr = c->PR;
  if ((e = launch(c, KK_BIN, b)) != cudaSuccess) return e;
  if (norm) {
    c->launches++;
    if ((e = dp_launch_norm(a, c->st)) != cudaSuccess) return e;
  }
  if (!last) return cudaSuccess;
  LaunchArgs x;
  x.p = c->p; x.st = c->st; x.ctr = c->ctrLL;
  x.n_pt_blocks = 0; x.apply_phi = 0; x.do_mu = 0; x.ll_bins = 1;
  x.grid = dim3(1);
  return launch(c, KK_XT, x);
}

fmnmf_status dp_err(fmnmf_dp* d, fmnmf_status s, const char* msg) {
  return set_err(d ? d->ctx : nullptr, s, "%s", msg);
}

}  // namespace

extern "C" {

fmnmf_status fmnmf_dp_default_opts(fmnmf_dp_opts* o) {
  if (!o) return set_err(nullptr, FMNMF_EINVAL, "opts is NULL");
  o->D = 16;
  o->Hd = 128;
  o->n_proposals = 30;
  o->eps = 1e-4f;
  o->normalise = 1;
  o->stream = nullptr;
  return FMNMF_OK;
}

fmnmf_status fmnmf_dp_create(fmnmf_dp** out, const void* X, int x_on_device, int F, int T, int M, int N, int K,
                             const fmnmf_dp_opts* opts) {
  if (!out) return set_err(nullptr, FMNMF_EINVAL, "out is NULL");
  *out = nullptr;
  fmnmf_dp_opts o;
  fmnmf_dp_default_opts(&o);
  if (opts) o = *opts;
  if (N < 1 || N > 8 || K < 1 || (N - 1) * K > 256)
    return set_err(nullptr, FMNMF_EINVAL, "FastMNMF-DP needs 1 <= N <= 8 and (N-1)*K <= 256 (N=%d K=%d)", N, K);
  if (o.D < 1 || o.D > 256 || o.Hd < 4 || o.Hd > 1024 || o.Hd % 4 != 0)
    return set_err(nullptr, FMNMF_EINVAL, "decoder shape D=%d Hd=%d (need 1 <= D <= 256, Hd a multiple of 4 in [4, 1024])", o.D, o.Hd);
  if (o.n_proposals < 0 || !(o.eps >= 0.f) || !std::isfinite(o.eps))
    return set_err(nullptr, FMNMF_EINVAL, "n_proposals must be >= 0 and eps finite and >= 0");
  fmnmf_opts co;
  fmnmf_default_opts(&co);
  co.source_model = FMNMF_SOURCE_FREE;
  co.normalise = o.normalise;
  co.stream = o.stream;
  fmnmf_ctx* ctx = nullptr;
  fmnmf_status s = fmnmf_init(&ctx, X, x_on_device, F, T, M, N, 1, 0, &co);
  if (s != FMNMF_OK) return s;
  auto fail = [&](fmnmf_status st, const char* fmt, auto... args) {
    set_err(nullptr, st, fmt, args...);
    fmnmf_destroy(ctx);
    return st;
  };
  if (!ctx->fused) return fail(FMNMF_EINVAL, "FastMNMF-DP: N*M=%d is too large for the per-bin kernel", N * M);
  int dev = 0, optin = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(FMNMF_ECUDA, "FastMNMF-DP: device query failed");
  fmnmf_dp* d = new fmnmf_dp;
  d->ctx = ctx;
  d->o = o;
  d->F = F; d->T = T; d->M = M; d->N = N; d->K = K;
  d->mh = dp_mh_plan(F, T, M, o.D, o.Hd, sms, (size_t)optin - 1024);
  if (d->mh.C == 0) {
    delete d;
    return fail(FMNMF_EINVAL, "FastMNMF-DP: F*M=%d too large to stage one frame in shared memory", F * M);
  }
  if (dp_prepare(ctx->maxm, d->mh) != cudaSuccess) {
    delete d;
    return fail(FMNMF_ECUDA, "FastMNMF-DP: shared-memory attribute failed");
  }
  const size_t Fs = F, Ts = T, Ds = o.D, Hs = o.Hd, Ss = o.n_proposals, nK = (size_t)(N - 1) * K;
  d->draw_iters = kDpDrawIters;
  const size_t counts[] = {Fs, Ts, Ts * Ds, Fs * Ts, nK * Fs, nK * Ts, Hs * Ds, Hs, Fs * Hs, Fs, (size_t)N * Fs,
                           kDpDrawIters * Ss * Ts * Ds, kDpDrawIters * Ss * Ts, Ss * Ts};
  float** dst[] = {&d->u, &d->v, &d->Z, &d->R, &d->Wn, &d->Hn, &d->W1, &d->b1, &d->W2, &d->b2, &d->nu,
                   &d->xi, &d->logu, &d->lg};
  size_t off[15], total = 0;
  for (int i = 0; i < 14; ++i) {
    off[i] = total;
    total += ((counts[i] * 4 + 255) / 256) * 256;
  }
  off[14] = total;
  total += 256;
  if (cudaMalloc(&d->buf, total) != cudaSuccess) {
    delete d;
    return fail(FMNMF_ENOMEM, "FastMNMF-DP: cudaMalloc of %zu bytes failed", total);
  }
  for (int i = 0; i < 14; ++i) *dst[i] = (float*)((char*)d->buf + off[i]);
  d->acc = (unsigned long long*)((char*)d->buf + off[14]);
  if (cudaMemsetAsync(d->acc, 0, 8, ctx->st) != cudaSuccess || cudaStreamSynchronize(ctx->st) != cudaSuccess) {
    cudaFree(d->buf);
    delete d;
    return fail(FMNMF_ECUDA, "FastMNMF-DP: counter reset failed");
  }
  *out = d;
  return FMNMF_OK;
}

const char* fmnmf_dp_last_error(const fmnmf_dp* d) { return d ? d->ctx->err.c_str() : g_thread_err.c_str(); }

fmnmf_status fmnmf_dp_set_decoder(fmnmf_dp* d, const float* W1, const float* b1, const float* W2, const float* b2) {
  if (!d) return set_err(nullptr, FMNMF_EINVAL, "dp is NULL");
  if (!W1 || !b1 || !W2 || !b2) return dp_err(d, FMNMF_EINVAL, "set_decoder needs W1, b1, W2 and b2");
  fmnmf_ctx* ctx = d->ctx;
  const size_t D = d->o.D, Hd = d->o.Hd, F = d->F;
  const struct { const float* src; float* dst; size_t n; } c[4] = {
      {W1, d->W1, Hd * D}, {b1, d->b1, Hd}, {W2, d->W2, F * Hd}, {b2, d->b2, F}};
  for (auto& e : c)
    for (size_t i = 0; i < e.n; ++i)
      if (!std::isfinite(e.src[i])) return dp_err(d, FMNMF_EINVAL, "decoder weights must be finite");
  CK(cudaStreamSynchronize(ctx->st));
  for (auto& e : c) CK(cudaMemcpyAsync(e.dst, e.src, e.n * 4, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  d->have_decoder = true;
  d->have_state = false;  // r = sigma^2(z) changes with the decoder: the state must be set again
  return FMNMF_OK;
}

fmnmf_status fmnmf_dp_set_state(fmnmf_dp* d, const float* Z, const float* u, const float* v, const float* W,
                                const float* H, const float* G, const void* Q) {
  if (!d) return set_err(nullptr, FMNMF_EINVAL, "dp is NULL");
  fmnmf_ctx* ctx = d->ctx;
  if (!d->have_decoder) return dp_err(d, FMNMF_EINVAL, "set_state: set the decoder first");
  const size_t F = d->F, T = d->T, M = d->M, D = d->o.D, nK = (size_t)(d->N - 1) * d->K;
  if (!Z || !u || !v || !G || !Q || (nK && (!W || !H))) return dp_err(d, FMNMF_EINVAL, "set_state: NULL argument");
  for (size_t i = 0; i < T * D; ++i)
    if (!std::isfinite(Z[i])) return dp_err(d, FMNMF_EINVAL, "z must be finite");
  auto pos = [](const float* a, size_t n) {
    for (size_t i = 0; i < n; ++i) if (!(a[i] > 0.f) || !std::isfinite(a[i])) return false;
    return true;
  };
  if (!pos(u, F) || !pos(v, T) || (nK && (!pos(W, nK * F) || !pos(H, nK * T))))
    return dp_err(d, FMNMF_EINVAL, "u, v, W and H must be finite and positive");
  std::vector<float4> Qx;
  fmnmf_status s = check_gq(ctx, G, Q, Qx);
  if (s != FMNMF_OK) return s;
  CK(cudaStreamSynchronize(ctx->st));
  CK(cudaMemcpyAsync(d->Z, Z, T * D * 4, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(d->u, u, F * 4, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(d->v, v, T * 4, cudaMemcpyHostToDevice, ctx->st));
  if (nK) {
    CK(cudaMemcpyAsync(d->Wn, W, nK * F * 4, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(d->Hn, H, nK * T * 4, cudaMemcpyHostToDevice, ctx->st));
  }
  CK(cudaMemcpyAsync(ctx->p.G, G, (size_t)d->N * F * M * 4, cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->p.Qx, Qx.data(), Qx.size() * sizeof(float4), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemsetAsync(ctx->p.status, 0, 4, ctx->st));
  CK(cudaMemsetAsync(d->acc, 0, 8, ctx->st));
  ctx->launches += d->N > 1 ? 2 : 1;
  CK(dp_launch_init(dp_args(d), ctx->st));
  CK(cudaStreamSynchronize(ctx->st));  // the host vector Qx goes out of scope
  if ((s = refresh_state(ctx)) != FMNMF_OK) return s;
  if ((s = check_status(ctx)) != FMNMF_OK) return s;
  d->have_state = true;
  return FMNMF_OK;
}

fmnmf_status fmnmf_dp_get_state(fmnmf_dp* d, float* Z, float* u, float* v, float* W, float* H, float* G, void* Q) {
  if (!d) return set_err(nullptr, FMNMF_EINVAL, "dp is NULL");
  fmnmf_ctx* ctx = d->ctx;
  const size_t F = d->F, T = d->T, M = d->M, D = d->o.D, nK = (size_t)(d->N - 1) * d->K;
  CK(cudaStreamSynchronize(ctx->st));
  if (Z) CK(cudaMemcpyAsync(Z, d->Z, T * D * 4, cudaMemcpyDeviceToHost, ctx->st));
  if (u) CK(cudaMemcpyAsync(u, d->u, F * 4, cudaMemcpyDeviceToHost, ctx->st));
  if (v) CK(cudaMemcpyAsync(v, d->v, T * 4, cudaMemcpyDeviceToHost, ctx->st));
  if (W && nK) CK(cudaMemcpyAsync(W, d->Wn, nK * F * 4, cudaMemcpyDeviceToHost, ctx->st));
  if (H && nK) CK(cudaMemcpyAsync(H, d->Hn, nK * T * 4, cudaMemcpyDeviceToHost, ctx->st));
  if (G) CK(cudaMemcpyAsync(G, ctx->p.G, (size_t)d->N * F * M * 4, cudaMemcpyDeviceToHost, ctx->st));
  if (Q) CK(cudaMemcpyAsync(Q, ctx->p.Qf, F * M * M * sizeof(float2), cudaMemcpyDeviceToHost, ctx->st));
  return check_status(ctx);
}

fmnmf_status fmnmf_dp_iterate(fmnmf_dp* d, int n_iter, const float* xi, const float* logu, int draws_on_device) {
  if (!d) return set_err(nullptr, FMNMF_EINVAL, "dp is NULL");
  fmnmf_ctx* ctx = d->ctx;
  if (n_iter < 0) return dp_err(d, FMNMF_EINVAL, "n_iter < 0");
  if (!d->have_state) return dp_err(d, FMNMF_EINVAL, "iterate: set the decoder and the state first");
  const size_t S = d->o.n_proposals, T = d->T, D = d->o.D;
  if (S && n_iter && (!xi || !logu)) return dp_err(d, FMNMF_EINVAL, "iterate: the Metropolis draws are NULL");
  sync_wait_limit(ctx);
  const size_t xs = S * T * D, ls = S * T;
  for (int i0 = 0; i0 < n_iter; i0 += d->draw_iters) {
    const int n = std::min(d->draw_iters, n_iter - i0);
    const float* xb = nullptr;
    const float* lb = nullptr;
    if (S) {
      if (draws_on_device) {
        xb = xi + i0 * xs;
        lb = logu + i0 * ls;
      } else {
        CK(cudaMemcpyAsync(d->xi, xi + i0 * xs, n * xs * 4, cudaMemcpyHostToDevice, ctx->st));
        CK(cudaMemcpyAsync(d->logu, logu + i0 * ls, n * ls * 4, cudaMemcpyHostToDevice, ctx->st));
        xb = d->xi;
        lb = d->logu;
      }
    }
    for (int i = 0; i < n; ++i)
      CK(enqueue_dp_iteration(d, S ? xb + i * xs : nullptr, S ? lb + i * ls : nullptr, i0 + i == n_iter - 1));
  }
  return FMNMF_OK;
}

fmnmf_status fmnmf_dp_metropolis(fmnmf_dp* d, const float* xi, const float* logu, int draws_on_device,
                                 float* loggamma, long long* accepted) {
  if (!d) return set_err(nullptr, FMNMF_EINVAL, "dp is NULL");
  fmnmf_ctx* ctx = d->ctx;
  if (!d->have_state) return dp_err(d, FMNMF_EINVAL, "metropolis: set the decoder and the state first");
  const size_t S = d->o.n_proposals, T = d->T, D = d->o.D;
  if (!S) return FMNMF_OK;
  if (!xi || !logu) return dp_err(d, FMNMF_EINVAL, "metropolis: the draws are NULL");
  CK(cudaStreamSynchronize(ctx->st));
  DpArgs a = dp_args(d);
  if (draws_on_device) {
    a.xi = xi;
    a.logu = logu;
  } else {
    CK(cudaMemcpyAsync(d->xi, xi, S * T * D * 4, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(d->logu, logu, S * T * 4, cudaMemcpyHostToDevice, ctx->st));
    a.xi = d->xi;
    a.logu = d->logu;
  }
  a.loggamma = d->lg;
  unsigned long long before = 0, after = 0;
  CK(cudaMemcpyAsync(&before, d->acc, 8, cudaMemcpyDeviceToHost, ctx->st));
  ctx->launches++;
  CK(dp_launch_mh(a, d->mh, ctx->st));
  CK(cudaMemcpyAsync(&after, d->acc, 8, cudaMemcpyDeviceToHost, ctx->st));
  if (loggamma) CK(cudaMemcpyAsync(loggamma, d->lg, S * T * 4, cudaMemcpyDeviceToHost, ctx->st));
  fmnmf_status s = check_status(ctx);
  if (accepted) *accepted = (long long)(after - before);
  return s;
}

fmnmf_status fmnmf_dp_sync(fmnmf_dp* d) {
  if (!d) return set_err(nullptr, FMNMF_EINVAL, "dp is NULL");
  return check_status(d->ctx);
}

fmnmf_status fmnmf_dp_loglik(fmnmf_dp* d, double* ll) {
  if (!d) return set_err(nullptr, FMNMF_EINVAL, "dp is NULL");
  return fmnmf_loglik(d->ctx, ll);
}

fmnmf_status fmnmf_dp_accepted(fmnmf_dp* d, long long* n) {
  if (!d || !n) return set_err(d ? d->ctx : nullptr, FMNMF_EINVAL, "NULL argument");
  fmnmf_ctx* ctx = d->ctx;
  unsigned long long a = 0;
  CK(cudaMemcpyAsync(&a, d->acc, 8, cudaMemcpyDeviceToHost, ctx->st));
  fmnmf_status s = check_status(ctx);
  *n = (long long)a;
  return s;
}

fmnmf_status fmnmf_dp_separate(fmnmf_dp* d, void* out, int out_on_device) {
  if (!d) return set_err(nullptr, FMNMF_EINVAL, "dp is NULL");
  return fmnmf_separate(d->ctx, out, out_on_device);
}

fmnmf_status fmnmf_dp_destroy(fmnmf_dp* d) {
  if (!d) return FMNMF_OK;
  if (d->ctx && d->ctx->st) cudaStreamSynchronize(d->ctx->st);
  if (d->buf) cudaFree(d->buf);
  fmnmf_status s = fmnmf_destroy(d->ctx);
  delete d;
  return s;
}

}  // extern "C"
