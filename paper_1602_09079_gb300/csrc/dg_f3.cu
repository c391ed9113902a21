// Fused FP32-mixed stage kernel of the degree-3 modal DG basis (order 4).
#define DG_K 3
#include "dg_fused_inst.cuh"
