// Launch parameters of the JPEG1 rasterisation kernels (M.6).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace jxlr {

// M.6.1.1 results per block (one scan direction each).
struct JpegCond {
  float* h_approx;            // [bh][bw]
  float* h_slope;
  uint8_t* has_h;
  float* v_approx;
  float* v_slope;
  uint8_t* has_v;
};

struct JpegCondArgs {
  const int16_t* coef;
  int bw, bh;
  float q_h, q_v;             // Q[1] / Q[0] and Q[8] / Q[0] (binary32)
  float max_gap, min_step;
  JpegCond out;
};

struct JpegIdctArgs {
  const int16_t* coef;        // [bh][bw][64], index 8u + v
  int bw, bh;
  float dq[64];               // Q[k] I(8,u) I(8,v) times the unscaled-IDCT scale
  float* plane;               // [8 bh][8 bw]
  int cond;                   // 1: replace coefficients 0, 1, 8 from c (M.6.1.1)
  JpegCond c;
  float m0, m1;               // Q[0] I(8,0)^2, and times the scale of frequency 1
};

struct JpegGabArgs {
  const float* src;           // [8 bh][8 bw]
  float* dst;
  int bw, bh;
  float w0n, w1n, w2n;        // J.4 weights normalised to sum 1
  float threshold;
  int limit;
};

struct JpegPlane {
  const float* data;
  int w, h;                   // plane size in samples
  int up_x, up_y;             // 2x upsampling along x / y (M.6.4)
};

struct JpegColorArgs {
  JpegPlane p[3];
  int ncomp;                  // 1 (grey) or 3 (YCbCr)
  int xs, ys;
  void* out;
  size_t stride;              // bytes per output row
  int dtype;                  // jxlr_out_dtype (F32_LINEAR, F16_LINEAR, U8_SRGB)
};

bool upload_jpeg_constants(const float* odd8, const float* odd4, float odd2);
void launch_jpeg_idct(const JpegIdctArgs& a, cudaStream_t s);
// M.6.1.1 plateau scans: one thread per block row, then one per block
// column; returns the number of launches.
int launch_jpeg_cond(const JpegCondArgs& a, cudaStream_t s);
void launch_jpeg_gab(const JpegGabArgs& a, cudaStream_t s);
void launch_jpeg_color(const JpegColorArgs& a, cudaStream_t s);

}  // namespace jxlr
