// Step kernels for stencil radius 4 (space order 8).
#define FD_R 4
#include "fd_step_inst.cuh"
