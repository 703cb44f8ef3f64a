// Channel bucket M <= 8.
#define FM_MAXM 8
#include "fm_kernels_inst.cuh"
