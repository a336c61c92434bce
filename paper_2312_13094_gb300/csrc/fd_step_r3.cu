// Step kernels for stencil radius 3 (space order 6).
#define FD_R 3
#include "fd_step_inst.cuh"
