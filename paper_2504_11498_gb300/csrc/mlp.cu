// Learned Newton seed (MLP) kernels -- placeholder translation unit.
#include "bspl_internal.cuh"
