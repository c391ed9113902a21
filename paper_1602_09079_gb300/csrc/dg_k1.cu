// Kernels and launchers of the degree-1 modal DG basis (order 2).
#define DG_K 1
#include "dg_inst.cuh"
