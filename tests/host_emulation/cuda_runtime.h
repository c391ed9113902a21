// cuda_runtime.h -- host stand-in for the runtime names the kernel headers
// mention (test infrastructure, used only by the host emulation).
#pragma once
#include "emu.h"
typedef int cudaError_t;
typedef void* cudaStream_t;
#define cudaSuccess 0
struct double2 {
  double x, y;
};
