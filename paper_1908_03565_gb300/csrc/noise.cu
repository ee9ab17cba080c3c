// K.5.2 pseudorandom channels of the noise synthesis.
//
// Per 256 x 256 group, eight generators run through the three channels
// row by row, one step per 16-sample segment.  A thread owns one generator
// for a chunk of 32 rows of one channel: it jumps its state to the chunk's
// first step with the GF(2) matrices of 2^b steps (the update is linear),
// then steps through the chunk, writing samples 2i and 2i+1 of every
// segment.  The jump replaces up to 12,288 dependent steps per generator by
// at most 14 matrix-vector products, so the work spreads over all SMs.
#include <cuda_runtime.h>

#include "internal.h"
#include "noise.h"

namespace jxlr {

namespace {

__constant__ uint64_t c_njump[kNoiseJumpLevels * 256];

constexpr int kGroup = 256;
constexpr int kChunkRows = 32;
constexpr int kChunks = kGroup / kChunkRows;

__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// One step: the two words exchanged, then the printed xorshift update; the
// output is taken where the draft prints it.
__device__ __forceinline__ uint64_t gen_step(uint64_t& s0, uint64_t& s1) {
  const uint64_t a = s1;
  uint64_t b = s0;
  b ^= b << 23;
  const uint64_t out = b + a;
  b ^= a ^ (b >> 18) ^ (a >> 5);
  s0 = a;
  s1 = b;
  return out;
}

// State after k steps (k < 2^kNoiseJumpLevels).
__device__ void gen_jump(uint64_t& s0, uint64_t& s1, int k) {
  for (int lv = 0; lv < kNoiseJumpLevels; ++lv) {
    if (!((k >> lv) & 1)) continue;
    const uint64_t* m = c_njump + lv * 256;
    uint64_t r0 = 0, r1 = 0;
#pragma unroll 8
    for (int j = 0; j < 64; ++j) {
      const uint64_t sel = 0ULL - ((s0 >> j) & 1ULL);
      r0 ^= m[2 * j] & sel;
      r1 ^= m[2 * j + 1] & sel;
    }
#pragma unroll 8
    for (int j = 0; j < 64; ++j) {
      const uint64_t sel = 0ULL - ((s1 >> j) & 1ULL);
      r0 ^= m[128 + 2 * j] & sel;
      r1 ^= m[128 + 2 * j + 1] & sel;
    }
    s0 = r0;
    s1 = r1;
  }
}

__global__ void __launch_bounds__(256) k_noise_gen(const __grid_constant__ NoiseGenArgs a) {
  const long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int gi = static_cast<int>(t & 7);
  const long long u = t >> 3;
  const int q = static_cast<int>(u % kChunks);
  const int c = static_cast<int>((u / kChunks) % 3);
  const long long g = u / (3 * kChunks);
  if (g >= static_cast<long long>(a.ngx) * a.ngy) return;
  const int gx = static_cast<int>(g % a.ngx), gy = static_cast<int>(g / a.ngx);
  const int x0 = gx * kGroup, y0 = gy * kGroup;
  const int w = min(kGroup, a.xs - x0), h = min(kGroup, a.ys - y0);
  const int r0 = q * kChunkRows;
  if (r0 >= h) return;
  const int nseg = (w + 15) >> 4;
  // K.5.2 seeding, generator gi
  const uint64_t seed = (static_cast<uint64_t>(y0) << 32) + static_cast<uint64_t>(x0);
  uint64_t s0 = splitmix64(seed + 0x9E3779B97F4A7C15ULL);
  uint64_t s1 = splitmix64(s0);
  for (int i = 1; i <= gi; ++i) {
    s0 = splitmix64(s1);
    s1 = splitmix64(s0);
  }
  gen_jump(s0, s1, (c * h + r0) * nseg);
  const int r1 = min(r0 + kChunkRows, h);
  for (int r = r0; r < r1; ++r) {
    float* row = a.r + c * a.ps + static_cast<size_t>(y0 + r) * a.rs + x0;
    for (int sgi = 0; sgi < nseg; ++sgi) {
      const uint64_t bits = gen_step(s0, s1);
      const int x = 16 * sgi + 2 * gi;
      const uint32_t lo = static_cast<uint32_t>(bits), hi = static_cast<uint32_t>(bits >> 32);
      if (x < w) row[x] = __uint_as_float((lo >> 9) | 0x3F800000u) - 1.f;
      if (x + 1 < w) row[x + 1] = __uint_as_float((hi >> 9) | 0x3F800000u) - 1.f;
    }
  }
}

}  // namespace

bool upload_noise_constants(const uint64_t* jump) {
  return cudaMemcpyToSymbol(c_njump, jump, sizeof(uint64_t) * kNoiseJumpLevels * 256) ==
         cudaSuccess;
}

int launch_noise_gen(const NoiseGenArgs& a, cudaStream_t s) {
  const long long threads = static_cast<long long>(a.ngx) * a.ngy * 3 * kChunks * 8;
  k_noise_gen<<<static_cast<unsigned>((threads + 255) / 256), 256, 0, s>>>(a);
  return 1;
}

}  // namespace jxlr
