// Kernel parameter blocks derived from the C-ABI parameters (shared by the
// context, batch paths).
#include <cmath>
#include <cstring>

#include "../../include/jxl_recon.h"
#include "internal.h"
#include "kernels.h"

namespace jxlr {

ColorParams color_params(const jxl_recon_filter_params& p) {
  ColorParams cp;
  const double div = p.target_nits_div50 * 50.0 / 250.0 * 255.0;
  for (int i = 0; i < 9; ++i) cp.m[i] = static_cast<float>(p.inv_opsin[i] / div);
  for (int i = 0; i < 3; ++i) cp.bias[i] = p.opsin_bias[i];
  return cp;
}

SigmaParams sigma_params(const jxl_recon_filter_params& p) {
  SigmaParams sp;
  const double im3 = std::cbrt(p.target_nits_div50 * 50.0 / 250.0);
  for (int c = 0; c < 3; ++c) {
    sp.gmin[c] = static_cast<float>((c == 0 ? -0.03 : 0.0) * im3);
    sp.gscale[c] = p.epf_scale[c];
  }
  sp.range_max = p.epf_range_max;
  sp.range_mul = p.epf_range_mul;
  sp.quant_mul = p.epf_quant_mul;
  sp.sigma_max = static_cast<float>(p.epf_sigma_max);
  for (int i = 0; i < 8; ++i) sp.lut[i] = p.epf_sharp_lut[i];
  return sp;
}

float one_minus_bias(int c) {
  // F.3: a quantised coefficient of magnitude <= 1 is scaled by 1 - kOneBias[c]
  static const double kOneBias[3] = {0.05465007330715401, 0.07005449891748593,
                                     0.049935103337343655};
  return static_cast<float>(1.0 - kOneBias[c]);
}

uint32_t weight_min_bits(float wmin) {
  // smallest binary32 value >= wmin (weights below it are dropped, J.2.5)
  if (!(wmin > 0)) return 0;
  uint32_t b;
  std::memcpy(&b, &wmin, 4);
  return b;
}

FilterArgs filter_args(const jxl_recon_filter_params& p) {
  FilterArgs f;
  std::memset(&f, 0, sizeof(f));
  f.epf = p.epf != 0;
  f.gab = p.gab != 0;
  for (int c = 0; c < 3; ++c) {
    const double w1 = p.gab_w1[c], w2 = p.gab_w2[c];
    const double n = 1.0 + 4.0 * w1 + 4.0 * w2;
    f.gw[c][0] = static_cast<float>(1.0 / n);
    f.gw[c][1] = static_cast<float>(w1 / n);
    f.gw[c][2] = static_cast<float>(w2 / n);
  }
  f.wmin_bits = weight_min_bits(p.epf_weight_min);
  f.sp = sigma_params(p);
  f.cp = color_params(p);
  f.noise = p.noise != 0;
  for (int k = 0; k < 16; ++k) f.noise_lut[k] = p.noise_lut[k];
  return f;
}

}  // namespace jxlr
