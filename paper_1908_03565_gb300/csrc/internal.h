// Internal declarations shared by the translation units of libjxlrecon.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/jxl_recon.h"

namespace jxlr {

constexpr int kNumCodes = 15;          // DctSelect codes 0..14 (C.5.4)
constexpr uint8_t kCovered = 0xFF;     // block covered by a varblock starting elsewhere
constexpr int kDequantFloats = 10560;  // sum over codes of 3 * W * H

enum Code : int {
  kDCT8 = 0, kIdentity = 1, kDCT2 = 2, kDCT4 = 3, kDCT16 = 4, kDCT32 = 5,
  kDCT16x8 = 6, kDCT8x16 = 7, kDCT32x8 = 8, kDCT8x32 = 9, kDCT32x16 = 10,
  kDCT16x32 = 11, kDCT4x8 = 12, kDCT8x4 = 13, kAFV = 14
};

// Width and height in samples of each code.  "DCT A x B" names A rows and B
// columns (C.6.1, I.2.3.5, I.2.3.6).
extern const int kShapeW[kNumCodes];
extern const int kShapeH[kNumCodes];

// Float offset of matrix (code, channel) inside a dequant table.
int dequant_offset(int code, int channel);

// C.6.1 default matrices, val = numerators / weights, [code][c][H][W]
// row-major in dequant_offset order.  Returns false if an entry outside the
// LLF slots is non-positive or not finite.
bool default_dequant(float* out /* kDequantFloats */);

// Multiplies a raw dequant table by the per-frequency scale of the draft's
// inverse transforms so the kernels can run unscaled cosine sums.
void prescale_dequant(const float* raw, float* scaled);

// Checks a caller table (C.6.1: non-positive or infinite entries are
// ill-formed).  LLF slots are not inspected.
bool dequant_valid(const float* table);

// I.2.7 LLF-from-DC maps for the DCT shapes, already multiplied by the
// transform scale: llf[j] = sum_i M[j][i] dc[i], j and i row-major over the
// cy x cx LLF block.  Index by llf_map_index(cx, cy); 16x16 floats each.
constexpr int kLlfMaps = 8;
int llf_map_index(int cx, int cy);
void llf_maps(float* out /* kLlfMaps * 256 */);
// The maps those invert (I.2.6 at N = 8 on the unscaled cosine basis):
// dc[i] = sum_j B[i][j] llf[j], B[i][j] at i * 16 + j, same index.
void llf_box_maps(float* out /* kLlfMaps * 256 */);

// Odd-part matrices of the unscaled N-point inverse DCT for N = 2..32:
// O_N[n][j] = cos((2n+1)(2j+1) pi / 2N), n, j < N/2, packed N = 32, 16, 8, 4, 2.
constexpr int kOddFloats = 256 + 64 + 16 + 4 + 1;
void odd_tables(float* out);

// Annex H maps on the unscaled cosine basis, for N = 8, 16, 32 packed in
// that order: up (N/4 x N/8 each, 42 floats) takes the N/8 DC samples of a
// varblock axis to the 4-sample means of its LLF-only reconstruction (I.2.6
// at N = 4); inv (N/4 x N/4 each, 84 floats) takes N/4 such means to the
// N/4 lowest coefficients (I.2.7 at N = 4, the exact inverse); half is the
// coefficient of 8-point frequency 1 whose 4-sample halves average to +-1
// (I.2.7.3 for DCT8x4 / DCT4x8).
constexpr int kLfUpFloats = 42;
constexpr int kLfInvFloats = 84;
void lf_tables(float* up, float* inv, float* half);

// K.5 generator jumps: for level b in [0, kNoiseJumpLevels), the 128 x 128
// GF(2) matrix of 2^b steps of one generator's state (s0 bits 0..63, then
// s1 bits 0..63), as 128 columns of (s0, s1) words.
constexpr int kNoiseJumpLevels = 14;
void noise_jump_tables(uint64_t* out /* kNoiseJumpLevels * 256 */);

// 4 * mul_table[sigma] of J.2.4 for sigma in [0, 672]; entries below 16 are 0.
void mul_table4(int32_t* out /* 673 */);

// Tensor-core basis tables: for N = 8 (padded to 16), 16, 32 at byte offsets
// 0, 1024, 2048, the FP16 hi then lo parts of B[n][k] = cos((2n+1)k pi/2N)
// in the canonical K-major no-swizzle operand layout (6144 bytes).
void tc_basis_tables(unsigned char* out);

// AFV basis of I.2.2, [coefficient][sample], 16 x 16.
extern const double kAfvBasis[16][16];

// Kernel parameter blocks from the C-ABI parameters (params.cpp).
struct ColorParams;
struct SigmaParams;
struct FilterArgs;
ColorParams color_params(const jxl_recon_filter_params& p);
SigmaParams sigma_params(const jxl_recon_filter_params& p);
uint32_t weight_min_bits(float wmin);
float one_minus_bias(int c);   // F.3, channel c
FilterArgs filter_args(const jxl_recon_filter_params& p);

// Context internals used by the batch path (api.cpp).
const float* ctx_default_dequant(const jxl_recon_ctx* c);
int ctx_device(const jxl_recon_ctx* c);
int ctx_precision(const jxl_recon_ctx* c);   // a jxlr_precision
int ctx_idle_slots(jxl_recon_ctx* c);   // slots without a request in flight
void ctx_count_launches(jxl_recon_ctx* c, int n);

// Resident CTAs per SM of the multi-image kernels (kernels.cu):
// kind 0 recon, 1 EPF (J.2 on the listed blocks), 2 Gaborish/colour, 3 its
// TMA form.
int batch_blocks_per_sm(int kind);

// Sets the message jxl_recon_last_error() returns on this thread (api.cpp).
void set_last_error(const std::string& msg);

// Device-side constant setup (kernels.cu): copies the tables above into
// __constant__ memory of the current device.
bool upload_constants(const float* llf, const float* box, const float* odd,
                      const int32_t* mul4, const float* afv);
// The same for the Annex H kernels (lf.cu).
bool upload_lf_constants(const float* up, const float* inv, float half);

}  // namespace jxlr
