// The fused step kernel instantiated with 16 threads per env (two envs per
// warp), in a translation unit of its own so that it compiles in parallel
// with the rest of the library.
#include "msh_fused.cuh"

FusedKernel fused_kernel_g16(int fl) { return fused_kernel_fl<256, 16>(fl); }
