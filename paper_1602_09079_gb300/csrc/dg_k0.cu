// Kernels and launchers of the degree-0 modal DG basis (order 1).
#define DG_K 0
#include "dg_inst.cuh"
