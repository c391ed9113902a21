// Fused FP32-mixed stage kernel of the degree-2 modal DG basis (order 3).
#define DG_K 2
#include "dg_fused_inst.cuh"
