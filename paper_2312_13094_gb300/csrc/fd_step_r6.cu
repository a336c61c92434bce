// Step kernels for stencil radius 6 (space order 12).
#define FD_R 6
#include "fd_step_inst.cuh"
