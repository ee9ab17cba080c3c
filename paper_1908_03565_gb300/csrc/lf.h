// Launch parameters of the DC-domain kernels (F.2 smoothing, Annex H).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace jxlr {

struct LfArgs {
  const int16_t* coef[3];
  size_t cstride;             // elements per coefficient row
  const uint8_t* vmap;        // [bh][bw]
  int bw, bh;
  size_t bpl;                 // bw * bh: floats per block-level plane
  float m_dc[3];
  float kx_dc, kb_dc;
  int smooth;                 // F.2 adaptive smoothing
  int predict;                // Annex H
  uint8_t* own;               // [bh][bw] scratch: code | dx << 4 | dy << 6, 0xFF none
  float* d1;                  // [3][bh][bw] out: DC after F.2 and G
  float* u;                   // [3][2bh][2bw] scratch: DC2x2 image (Annex H only)
  float* us;                  // [3][2bh][2bw] out: predicted W/4 x H/4 coefficients
};

// Enqueues the kernels on s; returns how many kernels it launched.
int launch_lf(const LfArgs& a, cudaStream_t s);

}  // namespace jxlr
