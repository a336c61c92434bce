// Step kernels for stencil radius 1 (space order 2).
#define FD_R 1
#include "fd_step_inst.cuh"
