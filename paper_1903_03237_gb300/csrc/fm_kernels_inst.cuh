// Instantiates the kernels of one channel bucket (FM_MAXM) and its launch entry points.
#include "fm_fused.cuh"
#include "fm_kernels.cuh"
#include "fm_launch.h"

#define FM_CAT2(a, b) a##b
#define FM_CAT(a, b) FM_CAT2(a, b)

namespace fm {

cudaError_t FM_CAT(launch_m, FM_MAXM)(KernelKind k, const LaunchArgs& a) {
  constexpr int MX = FM_MAXM;
  switch (k) {
    case KK_W: k_tile<MX, MODE_W><<<a.grid, kThreads, a.smem, a.st>>>(a.p, a.g, a.flags, a.ctr); break;
    case KK_H: k_tile<MX, MODE_H><<<a.grid, kThreads, a.smem, a.st>>>(a.p, a.g, a.flags, a.ctr); break;
    case KK_G: k_tile<MX, MODE_G><<<a.grid, kThreads, a.smem, a.st>>>(a.p, a.g, a.flags, a.ctr); break;
    case KK_Y: k_tile<MX, MODE_Y><<<a.grid, kThreads, a.smem, a.st>>>(a.p, a.g, a.flags, a.ctr); break;
    case KK_XT:
      k_xt_ll<MX><<<a.grid, kThreads, 0, a.st>>>(a.p, a.n_pt_blocks, a.apply_phi, a.do_mu, a.ctr, a.ll_bins, a.pr);
      break;
    case KK_PREP: k_prep_q<MX><<<a.grid, kThreads, 0, a.st>>>(a.p); break;
    case KK_SEP: k_separate<MX><<<a.grid, kThreads, a.smem, a.st>>>(a.p, a.g, a.out); break;
    case KK_IP:
      k_ip<MX><<<a.grid, MX * 32, a.smem, a.st>>>(a.p, a.S, a.flags, a.xt_mode, a.ctr, a.smem > 0 ? 1 : 0, a.pr, a.ll_tail);
      break;
    case KK_BIN: k_bin<MX><<<a.grid, kThreads, a.smem, a.st>>>(a.p, a.lam, a.pr, a.flags); break;
    case KK_HGEMM: {
      // cluster of a.g.S CTAs along z (the bin splits of one tile), set at launch
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = a.grid;
      cfg.blockDim = dim3(kThreads);
      cfg.dynamicSmemBytes = 0;
      cfg.stream = a.st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 1;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = (unsigned)a.g.S;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      return cudaLaunchKernelEx(&cfg, k_hgemm<MX>, a.p, (const float*)a.pr, a.g.span);
    }
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int FM_CAT(occupancy_m, FM_MAXM)(KernelKind k, size_t smem) {
  constexpr int MX = FM_MAXM;
  int n = 0;
  switch (k) {
    case KK_W: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tile<MX, MODE_W>, kThreads, smem); break;
    case KK_H: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tile<MX, MODE_H>, kThreads, smem); break;
    case KK_G: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tile<MX, MODE_G>, kThreads, smem); break;
    case KK_Y: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tile<MX, MODE_Y>, kThreads, smem); break;
    case KK_SEP: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_separate<MX>, kThreads, smem); break;
    default: n = 1;
  }
  return n > 0 ? n : 1;
}

int FM_CAT(occupancy_fused_m, FM_MAXM)(KernelKind k, size_t smem) {
  constexpr int MX = FM_MAXM;
  int n = 0;
  if (k == KK_BIN) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_bin<MX>, kThreads, smem);
  else if (k == KK_HGEMM) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_hgemm<MX>, kThreads, 0);
  return n;
}

cudaError_t FM_CAT(configure_m, FM_MAXM)(int bytes) {
  constexpr int MX = FM_MAXM;
  cudaError_t e = cudaSuccess;
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if ((e = cudaFuncSetAttribute(k_tile<MX, MODE_W>, A, bytes)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_tile<MX, MODE_H>, A, bytes)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_tile<MX, MODE_G>, A, bytes)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_tile<MX, MODE_Y>, A, bytes)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_separate<MX>, A, bytes)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_bin<MX>, A, bytes)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_ip<MX>, A, kIpPrefetchMax);
}

}  // namespace fm
