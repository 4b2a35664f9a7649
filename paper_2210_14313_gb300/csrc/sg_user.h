// Internal interface between the run-time compiled user integrands
// (sg_user.cu) and the entry points of sg_api.cu.
#pragma once
#include <cuda_runtime.h>

#include "../../include/sg.h"

#define SG_USER_MAX_STATE 16   // doubles of a user integrand's state
#define SG_USER_APAD 64        // prefix tuples per warp (as in sg_user_kernel.cuh)

// The compiled kernel of f, its state size and the device it was compiled for.
bool sg_integrand_kernel(sg_integrand f, cudaKernel_t *kern, int *K, int *device);
