// Launch parameters of the reconstruction kernels (device-side layout).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace jxlr {

// L.2 colour transform with the output scale folded in: rgb01 = m * mix,
// mix = gamma^3 + bias.
struct ColorParams {
  float m[9];
  float bias[3];
};

// J.2.2 guide and J.2.4 sigma parameters (binary32, the kernels' precision).
struct SigmaParams {
  float gmin[3];        // min[c] of J.2.2
  float gscale[3];      // epf_scale
  float range_max, range_mul, quant_mul, sigma_max;
  float lut[8];
};

struct OutParams {
  void* data;
  size_t stride;        // bytes per row
  int dtype;            // jxlr_out_dtype
};

// Work the sigma pass hands to the EPF (list == nullptr: none): the blocks
// with sigma >= 16 are appended to list (block indices), *count counting
// them; the others, which J.2 leaves unchanged, are copied to pass (the J.2
// output: planar XYB of the padded size, row / plane stride prs / pps in
// elements, 16-byte aligned rows).
struct EpfSink {
  int* list;
  unsigned* count;
  float* pass;
  size_t prs, pps;
};

struct ReconArgs {
  const int16_t* coef[3];
  size_t cstride;             // elements per coefficient row
  const uint8_t* vmap;        // [bh][bw]
  const float* acmul;         // [bh][bw]
  const float* cfl;           // [th][tw][2]
  const uint8_t* sharp;       // [bh][bw] (EPF only)
  const float* dequant;       // prescaled matrices, dequant_offset layout
  int xs, ys, wp, hp, bw, bh, tw;
  float m_dc[3];
  float kx_dc, kb_dc;
  float one_minus_bias[3];
  int write_xyb;              // 1: planar XYB to xyb; 0: final pixels to out
  float* xyb;                 // [3][hp][wp]
  int16_t* sigma;             // [bh][bw] or nullptr (no EPF)
  SigmaParams sp;
  ColorParams cp;
  OutParams out;
  const unsigned char* tcb;   // tensor-core basis tables (tensor-core variant only)
  unsigned* err;              // error flags of the tensor-core variant
  const float* dc1;           // [3][bh][bw] DC after F.2 smoothing and G, or nullptr
  const float* lfp;           // [3][2bh][2bw] Annex H coefficients, or nullptr
  EpfSink epf;                // with sigma
};

struct SigmaArgs {
  const float* xyb;
  size_t rstride, pstride;    // elements per row / per plane
  const uint8_t* vmap;
  const float* acmul;
  const uint8_t* sharp;
  int xs, ys, bw, bh;
  int16_t* sigma;
  SigmaParams sp;
  EpfSink epf;
};

struct FilterArgs {
  const float* xyb;
  size_t rstride, pstride;
  int xs, ys, bw;
  const int16_t* sigma;
  int epf, gab;
  float gw[3][3];             // Gaborish: centre, side, corner weights per channel
  uint32_t wmin_bits;         // smallest binary32 pattern with value >= epf_weight_min
  SigmaParams sp;             // guide parameters
  ColorParams cp;
  OutParams out;
  float* epf_out;             // J.2 result (planar XYB) of k_epf_work,
  size_t ors, ops;            // row / plane stride in elements
  const int* epf_list;        // multi-image J.2: the image's listed blocks and their
  const unsigned* epf_count;  // number (EpfSink of its sigma pass)
  unsigned* err;              // bounded device waits set bit 8 here on expiry (or nullptr)
  int noise;                  // K.5 after J.4: channels noise_r [3][ys][nrs]
  const float* noise_r;
  size_t nrs, nps;
  float noise_lut[16];
};

// J.3 on the EPF output f, in place, with the EPF input orig (planar XYB).
struct QcoArgs {
  const float* orig;
  size_t ors, ops;            // row / plane stride of orig (elements)
  float* f;
  size_t frs, fps;            // row / plane stride of f
  const uint8_t* vmap;        // [bh][bw]
  const float* acmul;         // [bh][bw]
  const float* dequant;       // prescaled matrices, dequant_offset layout
  int xs, ys, bw, bh;
  float m_dc[3];
  float mul;                  // qco_interval_mul
  int vec;                    // 1: both images allow 16-byte accesses of 8-sample chunks
};

void launch_validate(const uint8_t* vmap, int bw, int bh, unsigned* status, cudaStream_t s);
// Forms of the transform kernel: one CTA per 32x32 cell (grid), or a
// persistent grid of resident CTAs that fetch each next cell's
// coefficients and map during the current cell's stores.
enum { kReconGrid = 0, kReconPersistent = 1 };
void launch_recon(const ReconArgs& a, cudaStream_t s, int variant = kReconGrid);
// Variant whose separable passes of the varblocks larger than 8x8 run as
// FP16 hi/lo split products on the tensor cores (tcgen05, FP32 accumulate).
void launch_recon_tc(const ReconArgs& a, cudaStream_t s);
constexpr int kTcBasisBytes = 6144;
void launch_sigma(const SigmaArgs& a, cudaStream_t s);
void launch_qco(const QcoArgs& a, cudaStream_t s);
void launch_filter(const FilterArgs& a, cudaStream_t s);
// Gaborish / noise / colour (a.epf == 0) with the tile loaded by all threads
// (k_filter): no TMA and no bounded wait; same results bit for bit.
void launch_filter_plain(const FilterArgs& a, cudaStream_t s);
// J.2 on the blocks the sigma pass listed (EpfSink), into a.epf_out, where
// that pass copied the other blocks; J.4 / L.2 then run as launch_filter()
// on that output.  next: a zeroed counter the warps claim groups of 2 listed
// blocks from (or nullptr: a fixed round robin).
void launch_epf_work(const FilterArgs& a, const int* list, const unsigned* count, unsigned* next,
                     cudaStream_t s);

// Multi-image launches: args[i] per image (device array), prefix[i] = first
// work item of image i (prefix[nimg] = total), grid CTAs striding over items.
// The transform launch takes instead item_cell[2 w], item_cell[2 w + 1] =
// (image, cell index within it) of work item w.
void launch_recon_batch(const ReconArgs* args, const int* item_cell, int total, int grid,
                        cudaStream_t s);
void launch_filter_batch(const FilterArgs* args, const int* prefix, int nimg, int total, int grid,
                         cudaStream_t s);
// The TMA form of the multi-image Gaborish / colour launch: maps[i] is the
// tensor map of args[i].xyb made by make_filter_tensor_map() (kTensorMapBytes
// each, 64-byte aligned, in device memory); grid CTAs take the tiles
// round robin; bounded waits set bit 8 of *err on expiry.
constexpr size_t kTensorMapBytes = 128;
bool make_filter_tensor_map(const FilterArgs& a, void* tm);
void launch_filter_batch_tma(const FilterArgs* args, const int* prefix, const void* maps,
                             int nimg, int total, int grid, unsigned* err, cudaStream_t s);
// J.2 of many images (args[i].epf_list / epf_count / epf_out set; the sigma
// pass copied the unchanged blocks), persistent grid of one-warp CTAs;
// counts[i] is image i's listed-block count (args[i].epf_count == counts + i).
// next: a zeroed counter the warps claim the groups of all images from.
void launch_epf_work_batch(const FilterArgs* args, const unsigned* counts, int nimg, bool clamp,
                           int grid, unsigned* next, cudaStream_t s);
// Work items (32x32 tiles) of k_filter for a, and whether the EPF needs its
// exact-clamp variant for a's parameters.
int filter_tiles(const FilterArgs& a);
bool filter_needs_clamp(const FilterArgs& a);

}  // namespace jxlr
