// DC-domain steps ahead of the inverse transforms:
//   F.2  DC dequantisation and adaptive DC smoothing, then G for DC;
//   H    AC prediction from the DC2x2 image (with I.2.6 / I.2.7 at N = 4).
// The results are per-block DC samples (read by the reconstruction kernel in
// place of m_DC * q at the LLF slots) and a quarter-resolution plane of the
// predicted W/4 x H/4 coefficients (added to the dequantised coefficients
// outside the LLF corner).  Each kernel reads only inside its buffers
// whatever the DctSelect map holds.
#include <cuda_runtime.h>

#include "internal.h"
#include "lf.h"

namespace jxlr {

namespace {

__constant__ float c_lf_up[kLfUpFloats];
__constant__ float c_lf_inv[kLfInvFloats];
__constant__ float c_lf_half;

constexpr uint8_t kNoOwner = 0xFF;

// log2(W / 8) and log2(H / 8) of the DctSelect codes, two bits per code, so
// that lanes holding different codes look their shape up without a memory
// access (a constant-bank table serialises divergent lanes).
constexpr uint32_t shape_bits(bool width) {
  constexpr int lw[kNumCodes] = {0, 0, 0, 0, 1, 2, 0, 1, 0, 2, 1, 2, 0, 0, 0};
  constexpr int lh[kNumCodes] = {0, 0, 0, 0, 1, 2, 1, 0, 2, 0, 2, 1, 0, 0, 0};
  uint32_t m = 0;
  for (int i = 0; i < kNumCodes; ++i) m |= static_cast<uint32_t>(width ? lw[i] : lh[i]) << (2 * i);
  return m;
}
constexpr uint32_t kW8Bits = shape_bits(true), kH8Bits = shape_bits(false);
__device__ __forceinline__ int blocks_w(int code) { return 1 << ((kW8Bits >> (2 * code)) & 3); }
__device__ __forceinline__ int blocks_h(int code) { return 1 << ((kH8Bits >> (2 * code)) & 3); }

// Offsets of the N = 8, 16, 32 maps inside c_lf_up / c_lf_inv.
__device__ __forceinline__ int up_off(int N) { return N == 8 ? 0 : N == 16 ? 2 : 10; }
__device__ __forceinline__ int inv_off(int N) { return N == 8 ? 0 : N == 16 ? 4 : 20; }

__device__ __forceinline__ bool dct_shape(int code) {
  return code == 0 || (code >= 4 && code <= 11);
}

__device__ __forceinline__ int mirror1(int c, int size) {
  // 6.5 for coordinates at most one step outside [0, size)
  return c < 0 ? -c - 1 : c >= size ? 2 * size - 1 - c : c;
}

// Varblock owning block (bx, by): (code, dx, dy) packed as code | dx << 4 |
// dy << 6, or kNoOwner.  sv holds the map on the 12 x 12 blocks from
// (ox, oy).  Varblocks never cross a 32 x 32 cell (a map that makes them is
// rejected by validation), so the search stays in the block's cell;
// whatever the map holds, the result describes a varblock inside the image.
__device__ __forceinline__ int find_owner(const uint8_t (*sv)[12], int ox, int oy, int bw, int bh,
                                          int bx, int by) {
  for (int dy = 0; dy <= (by & 3); ++dy)
    for (int dx = 0; dx <= (bx & 3); ++dx) {
      const int code = sv[by - dy - oy][bx - dx - ox];
      if (code >= kNumCodes) continue;
      const int cx = blocks_w(code), cy = blocks_h(code);
      if (dx < cx && dy < cy && bx - dx + cx <= bw && by - dy + cy <= bh)
        return code | (dx << 4) | (dy << 6);
    }
  return kNoOwner;
}

// F.2 and G for one 32 x 32-sample cell (4 x 4 blocks), 64 threads: the raw
// DC samples of the cell and a 1-block ring (binary32, one rounding of
// q * m_DC, no extra levels), the smoothing window of F.2 on the cell's
// blocks (binary32, operation by operation in the order centre, edges
// N W E S, corners NW NE SW SE), then G for DC.  Writes the owner bytes and
// the DC samples of the cell's blocks and, for Annex H, the cell's 8 x 8
// DC2x2 samples: I.2.6 at N = 4 of each varblock from its DC samples alone.
__global__ void __launch_bounds__(64) k_dc_cell(const __grid_constant__ LfArgs a) {
  __shared__ float raw[3][6][6];
  __shared__ float dcs[3][4][4];
  __shared__ uint8_t own[4][4];
  __shared__ uint8_t sv[12][12];          // map of the 3 x 3 cells around this one
  __shared__ float s_up[kLfUpFloats];
  const int tid = threadIdx.x;
  const int cbx = 4 * blockIdx.x, cby = 4 * blockIdx.y;
  const int ox = cbx - 4, oy = cby - 4;
  for (int i = tid; i < 144; i += 64) {
    const int bx = ox + i % 12, by = oy + i / 12;
    sv[i / 12][i % 12] = (bx >= 0 && by >= 0 && bx < a.bw && by < a.bh)
                             ? __ldg(a.vmap + static_cast<size_t>(by) * a.bw + bx)
                             : kCovered;
  }
  if (tid < kLfUpFloats) s_up[tid] = c_lf_up[tid];
  __syncthreads();
  if (tid < 36) {
    const int bx = cbx - 1 + tid % 6, by = cby - 1 + tid / 6;
    float q[3] = {0.f, 0.f, 0.f};
    int o = kNoOwner;
    if (bx >= 0 && by >= 0 && bx < a.bw && by < a.bh) {
      o = find_owner(sv, ox, oy, a.bw, a.bh, bx, by);
      if (o != kNoOwner) {
        const int dx = (o >> 4) & 3, dy = o >> 6;
        const size_t at = static_cast<size_t>(8 * (by - dy) + dy) * a.cstride + 8 * (bx - dx) + dx;
        for (int c = 0; c < 3; ++c) q[c] = __fmul_rn(static_cast<float>(a.coef[c][at]), a.m_dc[c]);
      }
    }
    for (int c = 0; c < 3; ++c) raw[c][tid / 6][tid % 6] = q[c];
    const int lx = tid % 6 - 1, ly = tid / 6 - 1;
    if (lx >= 0 && lx < 4 && ly >= 0 && ly < 4) own[ly][lx] = static_cast<uint8_t>(o);
  }
  __syncthreads();
  if (tid < 16) {
    const int lx = tid & 3, ly = tid >> 2, bx = cbx + lx, by = cby + ly;
    float v[3];
    for (int c = 0; c < 3; ++c) {
      const float (*d)[6] = raw[c];
      const float s = d[ly + 1][lx + 1];
      v[c] = s;
      if (a.smooth && bx >= 1 && by >= 1 && bx + 1 < a.bw && by + 1 < a.bh) {
        const float edges = __fadd_rn(__fadd_rn(__fadd_rn(d[ly][lx + 1], d[ly + 1][lx]),
                                                d[ly + 1][lx + 2]), d[ly + 2][lx + 1]);
        const float corners = __fadd_rn(__fadd_rn(__fadd_rn(d[ly][lx], d[ly][lx + 2]),
                                                  d[ly + 2][lx]), d[ly + 2][lx + 2]);
        const float wa = __fadd_rn(__fadd_rn(__fmul_rn(0.05226273532324128f, s),
                                             __fmul_rn(0.20345139757231578f, edges)),
                                   __fmul_rn(0.0334829185968739f, corners));
        const float half = 0.5f * a.m_dc[c];
        if (__fsub_rn(s, half) <= wa && wa <= __fadd_rn(s, half)) v[c] = wa;
      }
    }
    v[0] = fmaf(a.kx_dc, v[1], v[0]);
    v[2] = fmaf(a.kb_dc, v[1], v[2]);
    if (bx < a.bw && by < a.bh) {
      const size_t o = static_cast<size_t>(by) * a.bw + bx;
      a.own[o] = own[ly][lx];
      for (int c = 0; c < 3; ++c) a.d1[c * a.bpl + o] = v[c];
    }
    for (int c = 0; c < 3; ++c) dcs[c][ly][lx] = v[c];
  }
  if (!a.predict) return;
  __syncthreads();
  // 8 x 8 DC2x2 samples, one per thread, three channels
  const int lx = tid & 7, ly = tid >> 3;
  const int x = 2 * cbx + lx, y = 2 * cby + ly;
  if (x >= 2 * a.bw || y >= 2 * a.bh) return;
  const int o = own[ly >> 1][lx >> 1];
  float val[3] = {0.f, 0.f, 0.f};
  if (o != kNoOwner) {
    const int code = o & 15, dx = (o >> 4) & 3, dy = o >> 6;
    const int cx = blocks_w(code), cy = blocks_h(code);
    const int vx = (lx >> 1) - dx, vy = (ly >> 1) - dy;      // varblock origin in the cell
    if (dct_shape(code) && cx * cy > 1 && vx >= 0 && vy >= 0 && vx + cx <= 4 && vy + cy <= 4) {
      const float* ax = s_up + up_off(8 * cx) + (2 * dx + (lx & 1)) * cx;
      const float* ay = s_up + up_off(8 * cy) + (2 * dy + (ly & 1)) * cy;
      for (int c = 0; c < 3; ++c) {
        float acc = 0.f;
        for (int p = 0; p < cy; ++p) {
          float t2 = 0.f;
          for (int q = 0; q < cx; ++q) t2 = fmaf(ax[q], dcs[c][vy + p][vx + q], t2);
          acc = fmaf(ay[p], t2, acc);
        }
        val[c] = acc;
      }
    } else {
      for (int c = 0; c < 3; ++c) val[c] = dcs[c][ly >> 1][lx >> 1];
    }
  }
  const size_t at = static_cast<size_t>(y) * (2 * a.bw) + x;
  for (int c = 0; c < 3; ++c) a.u[4 * c * a.bpl + at] = val[c];
}

// Annex H for one 32 x 32-sample cell (8 x 8 DC2x2 samples; a cell lies in
// one 256 x 256 group and holds whole varblocks), 128 threads:
//  1. the DC2x2 samples of the cell and a 1-sample ring: inside the group,
//     the DC2x2 image of k_dc_cell; outside the group (or the image), the DC
//     sample of the block that holds the position, mirrored at the image
//     bounds (the group's ring);
//  2. the smoothing window (0.12 / 0.2 / 0.02, |wa - s| <= 1.7 m_DC);
//  3. I.2.7 at N = 4: every DC2x2 position is one of the W/4 x H/4 lowest
//     coefficients of its varblock; those outside the LLF corner are
//     written to the prediction plane at that position.
__global__ void __launch_bounds__(128) k_lf_cell(const __grid_constant__ LfArgs a) {
  __shared__ float U[3][10][10];
  __shared__ float Us[3][8][8];
  __shared__ float s_inv[kLfInvFloats];
  const int tid = threadIdx.x;
  if (tid < kLfInvFloats) s_inv[tid] = c_lf_inv[tid];
  const int X0 = 8 * blockIdx.x, Y0 = 8 * blockIdx.y;     // cell origin in DC2x2 samples
  const int pw = 2 * a.bw, ph = 2 * a.bh;
  const int gx0 = X0 & ~63, gy0 = Y0 & ~63;
  const int gx1 = min(gx0 + 64, pw), gy1 = min(gy0 + 64, ph);

  for (int i = tid; i < 300; i += 128) {
    const int c = i / 100, t = i % 100;
    const int x = X0 - 1 + t % 10, y = Y0 - 1 + t / 10;
    float val;
    if (x >= gx0 && x < gx1 && y >= gy0 && y < gy1) {
      val = a.u[4 * c * a.bpl + static_cast<size_t>(y) * pw + x];
    } else {
      const int bx = mirror1(x >> 1, a.bw), by = mirror1(y >> 1, a.bh);
      val = a.d1[c * a.bpl + static_cast<size_t>(by) * a.bw + bx];
    }
    U[c][t / 10][t % 10] = val;
  }
  __syncthreads();

  for (int i = tid; i < 192; i += 128) {
    const int c = i >> 6, ly = (i >> 3) & 7, lx = i & 7;
    const float s = U[c][ly + 1][lx + 1];
    const float edges = (U[c][ly][lx + 1] + U[c][ly + 1][lx]) + (U[c][ly + 1][lx + 2] + U[c][ly + 2][lx + 1]);
    const float corners = (U[c][ly][lx] + U[c][ly][lx + 2]) + (U[c][ly + 2][lx] + U[c][ly + 2][lx + 2]);
    const float wa = fmaf(0.12f, s, fmaf(0.2f, edges, 0.02f * corners));
    const float t = 1.7f * a.m_dc[c];
    Us[c][ly][lx] = (s - t <= wa && wa <= s + t) ? wa : s;
  }
  __syncthreads();

  for (int i = tid; i < 192; i += 128) {
    const int c = i >> 6, ly = (i >> 3) & 7, lx = i & 7;
    const int x = X0 + lx, y = Y0 + ly;
    if (x >= pw || y >= ph) continue;
    const int bx = x >> 1, by = y >> 1;
    const int o = a.own[static_cast<size_t>(by) * a.bw + bx];
    if (o == kNoOwner) continue;
    const int code = o & 15, dx = (o >> 4) & 3, dy = o >> 6;
    const int cx = blocks_w(code), cy = blocks_h(code);
    const int nx = 2 * cx, ny = 2 * cy;
    const int lx0 = 2 * (bx - dx) - X0, ly0 = 2 * (by - dy) - Y0;   // varblock in the cell
    const int u = lx - lx0, v = ly - ly0;
    if ((u < cx && v < cy) || lx0 < 0 || ly0 < 0 || lx0 + nx > 8 || ly0 + ny > 8) continue;
    const float (*us)[8] = Us[c];
    float val;
    if (dct_shape(code)) {
      const float* bxm = s_inv + inv_off(8 * cx) + u * nx;
      const float* bym = s_inv + inv_off(8 * cy) + v * ny;
      val = 0.f;
      for (int r = 0; r < ny; ++r) {
        float t2 = 0.f;
        for (int q = 0; q < nx; ++q) t2 = fmaf(bxm[q], us[ly0 + r][lx0 + q], t2);
        val = fmaf(bym[r], t2, val);
      }
    } else {
      const float tl = us[ly0][lx0], tr = us[ly0][lx0 + 1];
      const float bl = us[ly0 + 1][lx0], br = us[ly0 + 1][lx0 + 1];
      float c01, c10, c11;   // coefficients (row 0, col 1), (row 1, col 0), (row 1, col 1)
      if (code == 13) {      // DCT8x4: 8-tall, 4-wide halves side by side
        c01 = 0.25f * ((tl + bl) - (tr + br));
        c10 = 0.5f * (tl - bl) * c_lf_half;
        c11 = 0.5f * (tr - br) * c_lf_half;
      } else if (code == 12) {   // DCT4x8: 4-tall, 8-wide halves stacked
        c10 = 0.25f * ((tl + tr) - (bl + br));
        c01 = 0.5f * (tl - tr) * c_lf_half;
        c11 = 0.5f * (bl - br) * c_lf_half;
      } else {               // AuxDCT2x2 of I.2.3.2 (Identity, DCT2, DCT4, AFV)
        c01 = 0.25f * ((tl + tr) - (bl + br));
        c10 = 0.25f * ((tl - tr) + (bl - br));
        c11 = 0.25f * ((tl - tr) - (bl - br));
      }
      val = v == 0 ? c01 : u == 0 ? c10 : c11;
    }
    a.us[c * 4 * a.bpl + static_cast<size_t>(y) * pw + x] = val;
  }
}

}  // namespace

bool upload_lf_constants(const float* up, const float* inv, float half) {
  for (int c = 0; c < kNumCodes; ++c)   // the packed shape bits agree with the shape table
    if (8 << ((kW8Bits >> (2 * c)) & 3) != kShapeW[c] || 8 << ((kH8Bits >> (2 * c)) & 3) != kShapeH[c])
      return false;
  return cudaMemcpyToSymbol(c_lf_up, up, sizeof(float) * kLfUpFloats) == cudaSuccess &&
         cudaMemcpyToSymbol(c_lf_inv, inv, sizeof(float) * kLfInvFloats) == cudaSuccess &&
         cudaMemcpyToSymbol(c_lf_half, &half, sizeof(float)) == cudaSuccess;
}

int launch_lf(const LfArgs& a, cudaStream_t s) {
  const dim3 cells((a.bw + 3) / 4, (a.bh + 3) / 4);
  k_dc_cell<<<cells, 64, 0, s>>>(a);
  if (!a.predict) return 1;
  k_lf_cell<<<cells, 128, 0, s>>>(a);
  return 2;
}

}  // namespace jxlr
