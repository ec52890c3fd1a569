// Fused row kernels for blocks of 2 columns.
#define XAMG_NV 2
#include "rows_inst.cuh"
