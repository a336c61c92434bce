// Step kernels for stencil radius 2 (space order 4).
#define FD_R 2
#include "fd_step_inst.cuh"
