// Channel bucket M <= 2.
#define FM_MAXM 2
#include "fm_kernels_inst.cuh"
