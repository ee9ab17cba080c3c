// JPEG1 direct rasterisation (M.6): dequantisation and IDCT per 8x8 block,
// block-conditional Gaborish, 2x linear chroma upsampling and YCbCr -> RGB.
//
//  k_jpeg_cond_rows / k_jpeg_cond_cols  M.6.1.1 plateau scans, one thread
//               per block row / column.
//  k_jpeg_idct  128 threads = 16 blocks x 8 rows.  A thread loads one
//               coefficient row (8 x int16, one 128-bit load), dequantises
//               it with the prescaled table and transforms it; the block's
//               transpose goes through shared memory within the warp (a
//               block's 8 rows are 8 lanes of one warp), then the column
//               transform and the row store.
//  k_jpeg_gab   one 8x8 block per 64-thread CTA: J.4 on the plane (mirrored
//               at its bounds), the M.6.3 count by __syncthreads_count, and
//               the block's smoothed or original samples.
//  k_jpeg_color one output pixel per thread: M.6.4 upsampling of the
//               subsampled planes evaluated at the pixel (separable linear,
//               weights 3/4 and 1/4), M.6.5, the output encoding.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "jpeg1.h"

namespace jxlr {

namespace {

// cos((2n+1) (2j+1) pi / 16), n, j < 4, and cos((2n+1) (2j+1) pi / 8), n, j < 2:
// the odd parts of the unscaled 8- and 4-point inverse DCT.
__constant__ float c_jodd8[16];
__constant__ float c_jodd4[4];
__constant__ float c_jodd2;   // cos(pi / 4)

// Unscaled 8-point inverse DCT: x_n = sum_k c_k cos((2n+1) k pi / 16).
__device__ __forceinline__ void idct8(float (&x)[8]) {
  // even part: 4-point on c0, c2, c4, c6
  const float e0 = x[0] + x[4] * c_jodd2, e1 = x[0] - x[4] * c_jodd2;
  const float o0 = x[2] * c_jodd4[0] + x[6] * c_jodd4[1];
  const float o1 = x[2] * c_jodd4[2] + x[6] * c_jodd4[3];
  const float ev[4] = {e0 + o0, e1 + o1, e1 - o1, e0 - o0};
  float od[4];
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) s = fmaf(x[2 * j + 1], c_jodd8[n * 4 + j], s);
    od[n] = s;
  }
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    x[n] = ev[n] + od[n];
    x[7 - n] = ev[n] - od[n];
  }
}

// M.6.1.1 along one line of n blocks (rows: step 1 block; columns: step bw
// blocks), in binary32, operation by operation (the comparisons decide which
// coefficients are replaced).  acx: index of the AC coefficient of the scan
// direction (1 horizontal, 8 vertical).
__device__ void cond_line(const int16_t* coef, int first, int stride, int n, int acx, float q,
                          float max_gap, float min_step, float* approx, float* slope,
                          uint8_t* has) {
  auto dc = [&](int i) { return static_cast<int>(coef[static_cast<size_t>(first + i * stride) * 64]); };
  auto ac = [&](int i) { return static_cast<int>(coef[static_cast<size_t>(first + i * stride) * 64 + acx]); };
  int x = 0;
  while (x < n) {
    const int d = dc(x);
    int end = x;
    bool zero = ac(x) == 0;
    while (end + 1 < n && dc(end + 1) == d) {
      ++end;
      zero = zero && ac(end) == 0;
    }
    const int start = x;
    x = end + 1;
    bool sane = false;
    float frm = 0.f, to = 0.f;
    if (zero && !(start == 0 && end == n - 1)) {
      const float cur = static_cast<float>(d);
      frm = start == 0 ? cur
                       : 0.5f * __fadd_rn(__fadd_rn(cur, static_cast<float>(dc(start - 1))),
                                          __fmul_rn(q, static_cast<float>(ac(start - 1))));
      to = end == n - 1 ? cur
                        : 0.5f * __fadd_rn(__fadd_rn(cur, static_cast<float>(dc(end + 1))),
                                           __fmul_rn(q, static_cast<float>(ac(end + 1))));
      sane = fabsf(__fsub_rn(to, cur)) <= max_gap && fabsf(__fsub_rn(cur, frm)) <= max_gap &&
             fabsf(__fsub_rn(to, frm)) > min_step;
    }
    const float ratio = sane ? __fdiv_rn(__fsub_rn(to, frm), static_cast<float>(end - start + 1)) : 0.f;
    for (int i = start; i <= end; ++i) {
      const size_t o = static_cast<size_t>(first + i * stride);
      has[o] = sane ? 1 : 0;
      approx[o] = sane ? __fadd_rn(frm, __fmul_rn(__fadd_rn(0.5f, static_cast<float>(i - start)), ratio)) : 0.f;
      slope[o] = sane ? -0.5f * ratio : 0.f;
    }
  }
}

__global__ void __launch_bounds__(128) k_jpeg_cond_rows(const __grid_constant__ JpegCondArgs a) {
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  if (y >= a.bh) return;
  cond_line(a.coef, y * a.bw, 1, a.bw, 1, a.q_h, a.max_gap, a.min_step, a.out.h_approx,
            a.out.h_slope, a.out.has_h);
}

__global__ void __launch_bounds__(128) k_jpeg_cond_cols(const __grid_constant__ JpegCondArgs a) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= a.bw) return;
  cond_line(a.coef, x, a.bw, a.bh, 8, a.q_v, a.max_gap, a.min_step, a.out.v_approx,
            a.out.v_slope, a.out.has_v);
}

__global__ void __launch_bounds__(128) k_jpeg_idct(const __grid_constant__ JpegIdctArgs a) {
  __shared__ float sT[16][8][9];
  const int tid = threadIdx.x;
  const int lb = tid >> 3, r = tid & 7;
  const int blk = blockIdx.x * 16 + lb;
  const int nblk = a.bw * a.bh;
  float x[8];
  if (blk < nblk) {
    const int4 raw = __ldg(reinterpret_cast<const int4*>(a.coef + static_cast<size_t>(blk) * 64 + 8 * r));
    const int16_t* h = reinterpret_cast<const int16_t*>(&raw);
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = static_cast<float>(h[j]) * a.dq[8 * r + j];
    if (a.cond && r < 2) {   // M.6.1.1: coefficients 0 and 1 (row 0), 8 (row 1)
      const bool hh = a.c.has_h[blk] != 0, vh = a.c.has_v[blk] != 0;
      if (r == 0) {
        float dcv = static_cast<float>(h[0]);
        if (hh && vh) dcv = 0.5f * __fadd_rn(a.c.h_approx[blk], a.c.v_approx[blk]);
        else if (hh) dcv = a.c.h_approx[blk];
        else if (vh) dcv = a.c.v_approx[blk];
        x[0] = dcv * a.m0;
        if (hh) x[1] = a.c.h_slope[blk] * a.m1;
      } else if (vh) {
        x[0] = a.c.v_slope[blk] * a.m1;
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = 0.f;
  }
  // row r holds the coefficients of vertical frequency r: transform along
  // the horizontal frequencies first
  idct8(x);
#pragma unroll
  for (int j = 0; j < 8; ++j) sT[lb][r][j] = x[j];
  __syncwarp();
  // column r: the vertical transform of horizontal position r
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = sT[lb][j][r];
  idct8(x);
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 8; ++j) sT[lb][j][r] = x[j];
  __syncwarp();
  if (blk < nblk) {
    const int by = blk / a.bw, bx = blk - by * a.bw;
    float* dst = a.plane + static_cast<size_t>(8 * by + r) * (8 * a.bw) + 8 * bx;
    reinterpret_cast<float4*>(dst)[0] = make_float4(sT[lb][r][0], sT[lb][r][1], sT[lb][r][2], sT[lb][r][3]);
    reinterpret_cast<float4*>(dst)[1] = make_float4(sT[lb][r][4], sT[lb][r][5], sT[lb][r][6], sT[lb][r][7]);
  }
}

__device__ __forceinline__ int mirror_plane(int c, int n) {
  // 6.5, for coordinates at most one step outside [0, n)
  return c < 0 ? -c - 1 : c >= n ? 2 * n - 1 - c : c;
}

__global__ void __launch_bounds__(64) k_jpeg_gab(const __grid_constant__ JpegGabArgs a) {
  const int bx = blockIdx.x, by = blockIdx.y;
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  const int w = 8 * a.bw, h = 8 * a.bh;
  const int x = 8 * bx + tx, y = 8 * by + ty;
  float acc_c = 0.f, acc_e = 0.f, acc_d = 0.f;
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) {
    const float* row = a.src + static_cast<size_t>(mirror_plane(y + dy, h)) * w;
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      const float v = __ldg(row + mirror_plane(x + dx, w));
      if (dx == 0 && dy == 0) acc_c += v;
      else if (dx == 0 || dy == 0) acc_e += v;
      else acc_d += v;
    }
  }
  const float s = fmaf(a.w2n, acc_d, fmaf(a.w1n, acc_e, a.w0n * acc_c));
  const float p = a.src[static_cast<size_t>(y) * w + x];
  const bool inner = tx >= 1 && tx < 7 && ty >= 1 && ty < 7;
  const int count = __syncthreads_count(inner && fabsf(p - s) > a.threshold);
  a.dst[static_cast<size_t>(y) * w + x] = count < a.limit ? s : p;
}

// M.6.4 source index and weight of the second tap for output index o of a
// 2x upsampled axis of n samples: o = 2i -> (i, i-1), o = 2i+1 -> (i, i+1),
// index -1 reading 1 and index n reading n-2.
__device__ __forceinline__ void up_taps(int o, int n, int& i0, int& i1) {
  i0 = o >> 1;
  int j = (o & 1) ? i0 + 1 : i0 - 1;
  if (j < 0) j = -j;
  if (j >= n) j = 2 * n - 2 - j;
  i1 = min(max(j, 0), n - 1);
}

__device__ __forceinline__ float sample_up(const JpegPlane& p, int x, int y) {
  const float* s = p.data;
  if (!p.up_x && !p.up_y) return s[static_cast<size_t>(y) * p.w + x];
  int x0 = x, x1 = x, y0 = y, y1 = y;
  if (p.up_x) up_taps(x, p.w, x0, x1);
  if (p.up_y) up_taps(y, p.h, y0, y1);
  const float* r0 = s + static_cast<size_t>(y0) * p.w;
  const float* r1 = s + static_cast<size_t>(y1) * p.w;
  // horizontal first (M.6.4), then vertical
  const float h0 = p.up_x ? fmaf(0.75f, r0[x0], 0.25f * r0[x1]) : r0[x0];
  if (!p.up_y) return h0;
  const float h1 = p.up_x ? fmaf(0.75f, r1[x0], 0.25f * r1[x1]) : r1[x0];
  return fmaf(0.75f, h0, 0.25f * h1);
}

__global__ void __launch_bounds__(256) k_jpeg_color(const __grid_constant__ JpegColorArgs a) {
  const int x = blockIdx.x * 32 + (threadIdx.x & 31);
  const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (x >= a.xs || y >= a.ys) return;
  float r, g, b;
  const float yv = sample_up(a.p[0], x, y) + 128.f;
  if (a.ncomp == 1) {
    r = g = b = yv;
  } else {
    const float cb = sample_up(a.p[1], x, y), cr = sample_up(a.p[2], x, y);
    r = fmaf(1.402f, cr, yv);
    g = fmaf(-0.71414f, cr, fmaf(-0.34414f, cb, yv));
    b = fmaf(1.772f, cb, yv);
  }
  char* row = static_cast<char*>(a.out) + static_cast<size_t>(y) * a.stride;
  if (a.dtype == 2) {   // u8: clamp, round half up
    uint8_t* o = reinterpret_cast<uint8_t*>(row) + 3 * x;
    o[0] = static_cast<uint8_t>(floorf(fminf(fmaxf(r, 0.f), 255.f) + 0.5f));
    o[1] = static_cast<uint8_t>(floorf(fminf(fmaxf(g, 0.f), 255.f) + 0.5f));
    o[2] = static_cast<uint8_t>(floorf(fminf(fmaxf(b, 0.f), 255.f) + 0.5f));
  } else if (a.dtype == 1) {
    __half* o = reinterpret_cast<__half*>(row) + 3 * x;
    o[0] = __float2half_rn(r * (1.f / 255.f));
    o[1] = __float2half_rn(g * (1.f / 255.f));
    o[2] = __float2half_rn(b * (1.f / 255.f));
  } else {
    float* o = reinterpret_cast<float*>(row) + 3 * x;
    o[0] = r * (1.f / 255.f);
    o[1] = g * (1.f / 255.f);
    o[2] = b * (1.f / 255.f);
  }
}

}  // namespace

bool upload_jpeg_constants(const float* odd8, const float* odd4, float odd2) {
  return cudaMemcpyToSymbol(c_jodd8, odd8, sizeof(float) * 16) == cudaSuccess &&
         cudaMemcpyToSymbol(c_jodd4, odd4, sizeof(float) * 4) == cudaSuccess &&
         cudaMemcpyToSymbol(c_jodd2, &odd2, sizeof(float)) == cudaSuccess;
}

void launch_jpeg_idct(const JpegIdctArgs& a, cudaStream_t s) {
  const int nblk = a.bw * a.bh;
  k_jpeg_idct<<<(nblk + 15) / 16, 128, 0, s>>>(a);
}

int launch_jpeg_cond(const JpegCondArgs& a, cudaStream_t s) {
  k_jpeg_cond_rows<<<(a.bh + 127) / 128, 128, 0, s>>>(a);
  k_jpeg_cond_cols<<<(a.bw + 127) / 128, 128, 0, s>>>(a);
  return 2;
}

void launch_jpeg_gab(const JpegGabArgs& a, cudaStream_t s) {
  k_jpeg_gab<<<dim3(a.bw, a.bh), 64, 0, s>>>(a);
}

void launch_jpeg_color(const JpegColorArgs& a, cudaStream_t s) {
  k_jpeg_color<<<dim3((a.xs + 31) / 32, (a.ys + 7) / 8), 256, 0, s>>>(a);
}

}  // namespace jxlr
