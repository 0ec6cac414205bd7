// Interface between the handle (msh.cu) and the depth-camera kernel
// (msh_render.cu): the device arrays of the scene the cameras see.
#pragma once
#include <cuda_runtime.h>

struct RenderScene {
  int E;
  const int* body_off;     // [E+1]
  const int* static_off;   // [E+1]
  const float4* bdims;     // per body (d0, d1, d2, shape as int bits); shape 0 sphere, 1 capsule, 2 box
  const float4* sworld;    // per static box 6 float4: centre, rotation rows with half extents in .w, AABB lo, hi
  const float* pos;        // [B][3]
  const float* quat;       // [B][4] (w, x, y, z)
};

struct RenderCams {
  int ncam, width, height;
  float focal, near_, far_;
  const int* body;         // [E][ncam] env-local mount body, -1 = world
  const float* pose;       // [E][ncam][7]
};

int msh_render_launch(const RenderScene& sc, const RenderCams& cm, float* depth, cudaStream_t s);
