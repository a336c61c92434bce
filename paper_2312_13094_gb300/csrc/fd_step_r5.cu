// Step kernels for stencil radius 5 (space order 10).
#define FD_R 5
#include "fd_step_inst.cuh"
