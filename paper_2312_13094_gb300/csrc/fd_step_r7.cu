// Step kernels for stencil radius 7 (space order 14).
#define FD_R 7
#include "fd_step_inst.cuh"
