// Channel bucket M <= 4.
#define FM_MAXM 4
#include "fm_kernels_inst.cuh"
