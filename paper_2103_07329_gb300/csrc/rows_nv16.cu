// Fused row kernels for blocks of 16 columns.
#define XAMG_NV 16
#include "rows_inst.cuh"
