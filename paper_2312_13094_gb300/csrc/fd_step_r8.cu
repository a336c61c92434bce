// Step kernels for stencil radius 8 (space order 16).
#define FD_R 8
#include "fd_step_inst.cuh"
