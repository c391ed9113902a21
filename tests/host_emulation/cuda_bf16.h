// cuda_bf16.h -- host stand-in (test infrastructure): the BF16 type and
// conversions the kernels use are defined by the host emulation.
#pragma once
#include "emu.h"
