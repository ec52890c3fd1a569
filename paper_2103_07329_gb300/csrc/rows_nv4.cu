// Fused row kernels for blocks of 4 columns.
#define XAMG_NV 4
#include "rows_inst.cuh"
