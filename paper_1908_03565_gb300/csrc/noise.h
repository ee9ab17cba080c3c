// Launch parameters of the K.5.2 generator kernel.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace jxlr {

struct NoiseGenArgs {
  float* r;                   // [3][ys][rs] pseudorandom channels RR, RG, RB
  size_t rs, ps;              // row / plane stride in elements
  int xs, ys;                 // image size (groups of 256 x 256 from the origin)
  int ngx, ngy;               // groups along x / y
};

bool upload_noise_constants(const uint64_t* jump);
int launch_noise_gen(const NoiseGenArgs& a, cudaStream_t s);

}  // namespace jxlr
