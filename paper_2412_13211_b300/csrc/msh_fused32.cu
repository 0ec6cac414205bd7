// The fused step kernel instantiated with 32 threads per env (one env per
// warp), in a translation unit of its own so that it compiles in parallel
// with the rest of the library.
#include "msh_fused.cuh"

FusedKernel fused_kernel_g32(int fl) { return fused_kernel_fl<256, 32>(fl); }
