// Host-side constant tables of the reconstruction path (double precision,
// rounded once to float for the device).
//
//  * dequantisation matrices: C.6.1 (numerators / weights), defaults C.6.1.1
//  * per-frequency scale of the inverse transforms: I.2.1 (N = 8) and the
//    Annex R generator (N = 2, 4, 16, 32); with the numerators' I(N, u) of
//    I.2.6.1 the composite is the orthonormal DCT-III basis
//  * LLF from DC: I.2.7, as the exact inverse of the 8x8 box mean of I.2.6
//  * mul_table: J.2.4 with kSigmaShift = 2
//  * AFV basis: I.2.2 (two rows printed with a surplus 0.0, repaired)
#include <cuda_fp16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace jxlr {

const int kShapeW[kNumCodes] = {8, 8, 8, 8, 16, 32, 8, 16, 8, 32, 16, 32, 8, 8, 8};
const int kShapeH[kNumCodes] = {8, 8, 8, 8, 16, 32, 16, 8, 32, 8, 32, 16, 8, 8, 8};

int dequant_offset(int code, int channel) {
  int off = 0;
  for (int k = 0; k < code; ++k) off += 3 * kShapeW[k] * kShapeH[k];
  return off + channel * kShapeW[code] * kShapeH[code];
}

namespace {

const double kPi = 3.14159265358979323846;

// ---- I.2.6.1 scaling helpers -------------------------------------------
double i8(int n, int u) {
  double eps = u == 0 ? std::sqrt(0.5) : 1.0;
  return std::sqrt(2.0 / n) * eps * std::cos(u * kPi / (2.0 * n));
}
double d8(int n, int u) { return 1.0 / (n * i8(n, u)); }
double scale_i(int n, int u) { return n == 8 ? i8(n, u) : d8(n, u); }

// Per-frequency scale of the draft's N-point inverse DCT relative to the
// unscaled cosine sum sum_k c_k cos((2n+1) k pi / 2N).
double idct_scale(int n, int k) {
  if (k == 0) return 1.0;
  if (n == 8) return 1.0 / std::cos(k * kPi / 16.0);
  return 2.0 * std::cos(k * kPi / (2.0 * n));
}

// ---- C.6.1 weights ------------------------------------------------------
double band_factor(double x) { return x > 0 ? x + 1.0 : 1.0 / (1.0 - x); }

// Geometric interpolation between bands; positions at or beyond the last
// band take the last band.
double interp(double pos, double vmax, const std::vector<double>& b) {
  const int len = static_cast<int>(b.size());
  double sp = pos * (len - 1) / vmax;
  int idx = static_cast<int>(std::floor(sp));
  if (idx >= len - 1) return b[len - 1];
  double fr = sp - idx;
  return b[idx] * std::pow(b[idx + 1] / b[idx], fr);
}

// Mode DCT weights for an X-wide, Y-tall matrix, out[y * X + x].
void dct_weights(int X, int Y, const double* db, int ndb, const double* eb, int neb,
                 double* out) {
  std::vector<double> dist(ndb), ecc(neb + 1);
  dist[0] = db[0];
  for (int i = 1; i < ndb; ++i) dist[i] = band_factor(db[i]) * dist[i - 1];
  ecc[0] = 1.0;
  for (int i = 0; i < neb; ++i) ecc[i + 1] = band_factor(eb[i]) * ecc[i];
  for (int y = 0; y < Y; ++y) {
    for (int x = 0; x < X; ++x) {
      double fx = double(x) / X, fy = double(y) / Y;
      double d = std::sqrt(fx * fx + fy * fy);
      double e = d > 0 ? std::fabs(fx - fy) / d : 0.0;
      out[y * X + x] = interp(d, std::sqrt(2.0), dist) * interp(e, 1.0, ecc);
    }
  }
}

// Default encodings (C.6.1.1), per channel X, Y, B.
const double kDbDct8[3][6] = {{5.0, 0.0, -0.4, -0.4, -0.4, -2.0},
                              {1.1, 0.0, -0.3, -0.3, -0.3, -0.3},
                              {1.0, -3.0, 0.0, 0.0, -1.0, -2.0}};
const double kIdentityParam[3][3] = {
    {221.50801256717435, 7087.151589594002, 4466.9924939259863},
    {29.535505378287006, 1454.6663024982124, 1368.041230099175},
    {9.2887405354132238, 23.982311358829531, 11.201853748207084}};
const double kDct2[3][6] = {{3840.0, 2560.0, 1280.0, 640.0, 480.0, 300.0},
                            {960.0, 640.0, 320.0, 180.0, 140.0, 120.0},
                            {640.0, 320.0, 128.0, 64.0, 32.0, 16.0}};
const double kDbDct4[3][4] = {
    {32.0, -0.4, 0.0, 0.0}, {6.0, 0.0, 0.0, -0.0}, {4.0, -5.0, -1.0, -1.0}};
const double kDct4Param[3][2] = {{1.0, 1.0}, {0.7, 0.7}, {1.0, 1.0}};
const double kDbDct16[3][7] = {
    {3.1965020925735868, -1.8000777393353804, -0.39424529824571225,
     -0.33909377445710343, -0.6350101832695744, -0.90177264050827612,
     -1.5162099239887414},
    {0.77917081615440487, -0.57424582104194355, -0.90745813428471001,
     -0.64925837484843441, -0.35865440981033403, -0.21322389111877305,
     -0.27615025315725483},
    {0.22259376988644336, -3.0531423165804414, -0.2, -0.30687130033378396,
     -0.42708730624733904, -1.4856834539296244, -5.9209142884401604}};
const double kDbDct32[3][8] = {
    {0.47968775359573942, -1.025, -0.98, -0.9012, -0.4, -0.48819395464,
     -0.421064, -0.27},
    {0.22295421389982905, -0.8041958212306401, -0.7633036457487539,
     -0.55660379990111464, -0.49785304658857626, -0.43699592683512467,
     -0.40180866526242109, -0.27321683125358037},
    {0.11607457694128877, -3.060733579805728, -2.0413270132490346,
     -2.0235650159727417, -0.5495389509954993, -0.4, -0.4, -0.3}};
const double kDbDct16x8[3][7] = {{5.0, -0.7, -0.7, -0.2, -0.2, -0.2, -0.5},
                                 {1.0, -0.5, -0.5, -0.5, -0.2, -0.2, -0.2},
                                 {0.35, -1.4, -0.2, -0.5, -0.5, -1.5, -3.6}};
const double kDbDct32x8[3][8] = {
    {0.90897201669289496, -2.523575079652864, 1.5606102630460328,
     -0.6828050717528521, -14.770016895841904, -31.365240527393656,
     0.565929254166433, 26.789646874558219},
    {0.3603042187746216, -0.11724474917749789, -0.85426302204085935,
     -0.5404181207241352, -0.45637619443533173, -0.82707923060149569,
     -1.09760551067614, -54.16057009483842},
    {0.25176400522276937, -10.060949304689093, -4.5316627381323995,
     -5.4569229849460807, -10.549754675878864, 1.7512906265092971,
     -1.6854706115725824, 3.3092762331901451}};
const double kEbDct32x8[3][4] = {
    {-0.40751133465833289, 2.2055690721475925, -1.4434547377534228,
     2.0590289434445102},
    {0.12452072219659419, 0.065578935001406033, -0.14598888885596958,
     0.12114139909222557},
    {0.0586589025020419, -2.2654958780302183, -4.6996221931893647,
     1.8254498073137184}};
const double kDbDct32x16[3][8] = {
    {1.1280371559733287, -0.98868, -0.658, -0.42026, -0.22712, -0.2206, -0.226,
     -0.2},
    {0.38961075971152237, -0.62525308982767058, -0.83770786552491361,
     -0.79014862079498627, -0.2692727459704829, -0.38272769465388551,
     -0.2292422253091453, -0.20719098826199578},
    {0.098, -2.41, -0.23, -0.2, -0.4, -0.8, -0.4, -0.5}};
const double kDbDct4x8[3][4] = {
    {17.142628543359718, -0.16269623020744692, -0.31194253026666783,
     -0.2151140670773547},
    {4.6225628588812384, -0.82630200888366945, -1.0675229603596517,
     -0.17845290869168118},
    {0.81188546639482984, -0.6594385811273854, -0.050082094097871593,
     -2.6843722511996204}};
const double kDct4x8Mult[3] = {1.0, 1.0, 1.0};
const double kAfvWeights[3][8] = {
    {6368.834817724610816928, 232.1096058872860158351, 415.663547479750900044,
     220.0720486370546864556, 329.818962738766012564, -0.9919974139384578, 0.0,
     -0.60},
    {1608.323575150649711025, 67.2724358236086, 89.06657498438612,
     64.07248898359674, 125.6541247697168638611, -2.2833978673775697, -0.14,
     -0.2485},
    {195.927828574730424638, 21.841306388764952, 18.5279466567289584105,
     12.573868715940659, 15.89916083965558, -0.41, -0.1608, 0.0}};
const double kAfvDct4Mult[3][2] = {{1.0, 1.0}, {1.0, 1.0}, {1.0, 1.0}};
const double kAfvFreqs[16] = {0.0, 0.0, 0.8517778890324296, 5.37778436506804,
                              0.0, 0.0, 4.734747904497923, 5.449245381693219,
                              1.6598270267479331, 4.0, 7.275749096817861,
                              10.423227632456525, 2.662932286148962,
                              7.630657783650829, 8.962388608184032,
                              12.97166202570235};
const double kAfvLo = 0.8517778890324296;
const double kAfvHi = 12.1198851366699204;

// weights[y * W + x] of (code, channel).
void weights(int code, int c, double* w) {
  const double zero4[4] = {0, 0, 0, 0};
  const int W = kShapeW[code], H = kShapeH[code];
  switch (code) {
    case kDCT8: dct_weights(8, 8, kDbDct8[c], 6, zero4, 3, w); return;
    case kDCT16: dct_weights(16, 16, kDbDct16[c], 7, zero4, 3, w); return;
    case kDCT32: dct_weights(32, 32, kDbDct32[c], 8, zero4, 4, w); return;
    case kDCT16x8: case kDCT8x16: dct_weights(W, H, kDbDct16x8[c], 7, zero4, 3, w); return;
    case kDCT32x8: case kDCT8x32: dct_weights(W, H, kDbDct32x8[c], 8, kEbDct32x8[c], 4, w); return;
    case kDCT32x16: case kDCT16x32: dct_weights(W, H, kDbDct32x16[c], 8, zero4, 4, w); return;
    case kIdentity:
      for (int i = 0; i < 64; ++i) w[i] = kIdentityParam[c][0];
      w[1] = w[8] = kIdentityParam[c][1];
      w[9] = kIdentityParam[c][2];
      return;
    case kDCT2:
      for (int y = 0; y < 8; ++y) {
        for (int x = 0; x < 8; ++x) {
          int m = x > y ? x : y;   // Chebyshev ring of (x, y)
          int lo = x < y ? x : y;
          double v;
          if (m >= 4) v = lo >= 4 ? kDct2[c][5] : kDct2[c][4];
          else if (m >= 2) v = lo >= 2 ? kDct2[c][3] : kDct2[c][2];
          else if (m == 1) v = lo == 1 ? kDct2[c][1] : kDct2[c][0];
          else v = 1.0;  // (0, 0): LLF slot, never used
          w[y * 8 + x] = v;
        }
      }
      return;
    case kDCT4: {
      double w4[16];
      dct_weights(4, 4, kDbDct4[c], 4, zero4, 2, w4);
      for (int y = 0; y < 8; ++y)
        for (int x = 0; x < 8; ++x) w[y * 8 + x] = w4[(y / 2) * 4 + x / 2];
      w[1] /= kDct4Param[c][0];
      w[8] /= kDct4Param[c][0];
      w[9] /= kDct4Param[c][1];
      return;
    }
    case kDCT4x8: case kDCT8x4: {
      double w84[32];  // 8 wide, 4 tall
      dct_weights(8, 4, kDbDct4x8[c], 4, zero4, 2, w84);
      double t[64];
      for (int y = 0; y < 8; ++y)
        for (int x = 0; x < 8; ++x) t[y * 8 + x] = w84[(y / 2) * 8 + x];
      t[8] /= kDct4x8Mult[c];   // (x = 0, y = 1)
      for (int y = 0; y < 8; ++y)
        for (int x = 0; x < 8; ++x)
          w[y * 8 + x] = code == kDCT4x8 ? t[y * 8 + x] : t[x * 8 + y];
      return;
    }
    case kAFV: {
      const double* aw = kAfvWeights[c];
      std::vector<double> bands(4);
      bands[0] = aw[4];
      for (int i = 1; i < 4; ++i) bands[i] = bands[i - 1] * band_factor(aw[i + 4]);
      auto set = [&](int x, int y, double v) {
        for (int dy = 0; dy < 2; ++dy)
          for (int dx = 0; dx < 2; ++dx) w[(2 * y + dy) * 8 + 2 * x + dx] = v;
      };
      set(0, 0, aw[0]);
      set(0, 1, aw[1]);
      set(1, 0, aw[2]);
      set(1, 1, aw[3]);
      for (int y = 0; y < 4; ++y)
        for (int x = 0; x < 4; ++x)
          if (x >= 2 || y >= 2) set(x, y, interp(kAfvFreqs[y * 4 + x] - kAfvLo, kAfvHi, bands));
      w[1] *= kAfvDct4Mult[c][0];
      w[8] *= kAfvDct4Mult[c][0];
      w[9] *= kAfvDct4Mult[c][1];
      return;
    }
  }
}

// numerators[y * W + x] (C.6.1): I(N, f) per DCT dimension divided by the
// coefficient count; a 4-point dimension of a 64-entry matrix uses
// I(4, f / 2); modes DCT2, Identity and AFV use 1.
void numerators(int code, double* n) {
  const int W = kShapeW[code], H = kShapeH[code];
  for (int y = 0; y < H; ++y) {
    for (int x = 0; x < W; ++x) {
      double fx, fy;
      switch (code) {
        case kIdentity: case kDCT2: case kAFV: n[y * W + x] = 1.0; continue;
        case kDCT4: fx = scale_i(4, x / 2); fy = scale_i(4, y / 2); break;
        case kDCT4x8: fx = scale_i(8, x); fy = scale_i(4, y / 2); break;
        case kDCT8x4: fx = scale_i(4, x / 2); fy = scale_i(8, y); break;
        default: fx = scale_i(W, x); fy = scale_i(H, y); break;
      }
      n[y * W + x] = fx * fy / (W * H);
    }
  }
}

// Unscaled-cosine prescale of position (x, y) of a code's matrix.
double position_scale(int code, int x, int y) {
  const int W = kShapeW[code], H = kShapeH[code];
  switch (code) {
    case kIdentity: case kDCT2: case kAFV: return 1.0;
    case kDCT4: return idct_scale(4, x / 2) * idct_scale(4, y / 2);
    case kDCT4x8: return idct_scale(8, x) * idct_scale(4, y / 2);
    case kDCT8x4: return idct_scale(4, x / 2) * idct_scale(8, y);
    default: return idct_scale(W, x) * idct_scale(H, y);
  }
}

bool is_llf(int code, int x, int y) {
  return x < kShapeW[code] / 8 && y < kShapeH[code] / 8;
}

// Gauss-Jordan inverse of an n x n matrix (n <= 16), in place.
bool invert(double* a, int n) {
  std::vector<double> inv(n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(a[r * n + col]) > std::fabs(a[piv * n + col])) piv = r;
    if (std::fabs(a[piv * n + col]) < 1e-300) return false;
    for (int k = 0; k < n; ++k) {
      std::swap(a[col * n + k], a[piv * n + k]);
      std::swap(inv[col * n + k], inv[piv * n + k]);
    }
    double d = a[col * n + col];
    for (int k = 0; k < n; ++k) { a[col * n + k] /= d; inv[col * n + k] /= d; }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double f = a[r * n + col];
      if (f == 0) continue;
      for (int k = 0; k < n; ++k) {
        a[r * n + k] -= f * a[col * n + k];
        inv[r * n + k] -= f * inv[col * n + k];
      }
    }
  }
  std::memcpy(a, inv.data(), sizeof(double) * n * n);
  return true;
}

}  // namespace

const double kAfvBasis[16][16] = {
    {0.25, 0.25, 0.25, 0.25, 0.25, 0.25, 0.25, 0.25, 0.25, 0.25, 0.25, 0.25,
     0.25, 0.25, 0.25, 0.25},
    {0.876902929799142, 0.2206518106944235, -0.10140050393753763,
     -0.1014005039375375, 0.2206518106944236, -0.10140050393753777,
     -0.10140050393753772, -0.10140050393753763, -0.10140050393753758,
     -0.10140050393753769, -0.1014005039375375, -0.10140050393753768,
     -0.10140050393753768, -0.10140050393753759, -0.10140050393753763,
     -0.10140050393753741},
    {0.0, 0.0, 0.40670075830260755, 0.44444816619734445, 0.0, 0.0,
     0.19574399372042936, 0.2929100136981264, -0.40670075830260716,
     -0.19574399372042872, 0.0, 0.11379074460448091, -0.44444816619734384,
     -0.29291001369812636, -0.1137907446044814, 0.0},
    {0.0, 0.0, -0.2125574805828748, 0.3085497062849767, 0.0, 0.4706702258572536,
     -0.1621205195722993, 0.0, -0.21255748058287047, -0.16212051957228327,
     -0.47067022585725277, -0.1464291867126764, 0.3085497062849487, 0.0,
     -0.1464291867126536, 0.4251149611657548},
    // printed with 17 entries; one surplus trailing 0.0 dropped
    {0.0, -0.7071067811865474, 0.0, 0.0, 0.7071067811865476, 0.0, 0.0, 0.0,
     0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0},
    {-0.4105377591765233, 0.6235485373547691, -0.06435071657946274,
     -0.06435071657946266, 0.6235485373547694, -0.06435071657946284,
     -0.0643507165794628, -0.06435071657946274, -0.06435071657946272,
     -0.06435071657946279, -0.06435071657946266, -0.06435071657946277,
     -0.06435071657946277, -0.06435071657946273, -0.06435071657946274,
     -0.0643507165794626},
    {0.0, 0.0, -0.4517556589999482, 0.15854503551840063, 0.0,
     -0.04038515160822202, 0.0074182263792423875, 0.39351034269210167,
     -0.45175565899994635, 0.007418226379244351, 0.1107416575309343,
     0.08298163094882051, 0.15854503551839705, 0.3935103426921022,
     0.0829816309488214, -0.45175565899994796},
    {0.0, 0.0, -0.304684750724869, 0.5112616136591823, 0.0, 0.0,
     -0.290480129728998, -0.06578701549142804, 0.304684750724884,
     0.2904801297290076, 0.0, -0.23889773523344604, -0.5112616136592012,
     0.06578701549142545, 0.23889773523345467, 0.0},
    {0.0, 0.0, 0.3017929516615495, 0.25792362796341184, 0.0,
     0.16272340142866204, 0.09520022653475037, 0.0, 0.3017929516615503,
     0.09520022653475055, -0.16272340142866173, -0.35312385449816297,
     0.25792362796341295, 0.0, -0.3531238544981624, -0.6035859033230976},
    // printed with 17 entries; the 0.0 at index 3 dropped
    {0.0, 0.0, 0.40824829046386274, 0.0, 0.0, 0.0, 0.0, -0.4082482904638628,
     -0.4082482904638635, 0.0, 0.0, -0.40824829046386296, 0.0,
     0.408248290463863, 0.408248290463863, 0.0},
    {0.0, 0.0, 0.1747866975480809, 0.0812611176717539, 0.0, 0.0,
     -0.3675398009862027, -0.307882213957909, -0.17478669754808135,
     0.3675398009862011, 0.0, 0.4826689115059883, -0.08126111767175039,
     0.30788221395790305, -0.48266891150598584, 0.0},
    {0.0, 0.0, -0.21105601049335784, 0.18567180916109802, 0.0, 0.0,
     0.49215859013738733, -0.38525013709251915, 0.21105601049335806,
     -0.49215859013738905, 0.0, 0.17419412659916217, -0.18567180916109904,
     0.3852501370925211, -0.1741941265991621, 0.0},
    {0.0, 0.0, -0.14266084808807264, -0.3416446842253372, 0.0,
     0.7367497537172237, 0.24627107722075148, -0.08574019035519306,
     -0.14266084808807344, 0.24627107722075137, 0.14883399227113567,
     -0.04768680350229251, -0.3416446842253373, -0.08574019035519267,
     -0.047686803502292804, -0.14266084808807242},
    {0.0, 0.0, -0.13813540350758585, 0.3302282550303788, 0.0,
     0.08755115000587084, -0.07946706605909573, -0.4613374887461511,
     -0.13813540350758294, -0.0794670660591026, 0.49724647109535086,
     0.12538059448563663, 0.3302282550303805, -0.4613374887461554,
     0.12538059448564315, -0.13813540350758452},
    {0.0, 0.0, -0.1743760259965106, 0.0702790691196284, 0.0,
     -0.2921026642334881, 0.3623817333531167, 0.0, -0.1743760259965108,
     0.36238173335311646, 0.29210266423348785, -0.4326608024727445,
     0.07027906911962818, 0.0, -0.4326608024727457, 0.34875205199302267},
    {0.0, 0.0, 0.1135498731499337, -0.07417504595810355, 0.0,
     0.19402893032594343, -0.435190496523228, 0.21918684838857466,
     0.11354987314994257, -0.4351904965232251, 0.5550443808910661,
     -0.25468277124066463, -0.07417504595810233, 0.2191868483885728,
     -0.25468277124066413, 0.1135498731499429}};

bool default_dequant(float* out) {
  bool ok = true;
  std::vector<double> w(1024), n(1024);
  for (int code = 0; code < kNumCodes; ++code) {
    const int W = kShapeW[code], H = kShapeH[code];
    numerators(code, n.data());
    for (int c = 0; c < 3; ++c) {
      weights(code, c, w.data());
      float* dst = out + dequant_offset(code, c);
      for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
          double v = n[y * W + x] / w[y * W + x];
          if (!is_llf(code, x, y) && !(v > 0 && std::isfinite(v))) ok = false;
          dst[y * W + x] = static_cast<float>(v);
        }
      }
    }
  }
  return ok;
}

bool dequant_valid(const float* table) {
  for (int code = 0; code < kNumCodes; ++code) {
    const int W = kShapeW[code], H = kShapeH[code];
    for (int c = 0; c < 3; ++c) {
      const float* m = table + dequant_offset(code, c);
      for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
          if (!is_llf(code, x, y) && !(m[y * W + x] > 0 && std::isfinite(m[y * W + x])))
            return false;
    }
  }
  return true;
}

void prescale_dequant(const float* raw, float* scaled) {
  for (int code = 0; code < kNumCodes; ++code) {
    const int W = kShapeW[code], H = kShapeH[code];
    for (int c = 0; c < 3; ++c) {
      const int off = dequant_offset(code, c);
      for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
          scaled[off + y * W + x] =
              static_cast<float>(double(raw[off + y * W + x]) * position_scale(code, x, y));
    }
  }
}

namespace {
// Mean of the unscaled cosine f_k(n) = cos((2n+1) k pi / 2N) over n in
// [s, s + len).
double cos_mean(int N, int k, int s, int len) {
  double acc = 0;
  for (int n = s; n < s + len; ++n) acc += std::cos((2 * n + 1) * k * kPi / (2.0 * N));
  return acc / len;
}
}  // namespace

void lf_tables(float* up, float* inv, float* half) {
  int uo = 0, io = 0;
  for (int N = 8; N <= 32; N *= 2) {
    const int n4 = N / 4, n8 = N / 8;
    // M8[b][k]: 8-sample means of the LLF frequencies; M4L[q][k]: 4-sample
    // means of the same; M4[q][k]: 4-sample means of the N/4 LF frequencies.
    std::vector<double> m8(n8 * n8), m4(n4 * n4);
    for (int b = 0; b < n8; ++b)
      for (int k = 0; k < n8; ++k) m8[b * n8 + k] = cos_mean(N, k, 8 * b, 8);
    for (int q = 0; q < n4; ++q)
      for (int k = 0; k < n4; ++k) m4[q * n4 + k] = cos_mean(N, k, 4 * q, 4);
    invert(m8.data(), n8);
    for (int q = 0; q < n4; ++q)
      for (int b = 0; b < n8; ++b) {
        double acc = 0;
        for (int k = 0; k < n8; ++k) acc += cos_mean(N, k, 4 * q, 4) * m8[k * n8 + b];
        up[uo + q * n8 + b] = static_cast<float>(acc);
      }
    invert(m4.data(), n4);
    for (int i = 0; i < n4 * n4; ++i) inv[io + i] = static_cast<float>(m4[i]);
    uo += n4 * n8;
    io += n4 * n4;
  }
  *half = static_cast<float>(1.0 / cos_mean(8, 1, 0, 4));
}

namespace {
// One step of the K.5 generator's state (the two words exchanged, then the
// printed xorshift update); linear over GF(2).
void noise_state_step(uint64_t& s0, uint64_t& s1) {
  const uint64_t a = s1;
  uint64_t b = s0;
  b ^= b << 23;
  b ^= a ^ (b >> 18) ^ (a >> 5);
  s0 = a;
  s1 = b;
}
}  // namespace

void noise_jump_tables(uint64_t* out) {
  // level 0: the images of the 128 basis vectors under one step
  std::vector<uint64_t> cur(256), nxt(256);
  for (int j = 0; j < 128; ++j) {
    uint64_t s0 = j < 64 ? (1ULL << j) : 0, s1 = j < 64 ? 0 : (1ULL << (j - 64));
    noise_state_step(s0, s1);
    cur[2 * j] = s0;
    cur[2 * j + 1] = s1;
  }
  for (int lv = 0; lv < kNoiseJumpLevels; ++lv) {
    std::memcpy(out + lv * 256, cur.data(), sizeof(uint64_t) * 256);
    // square: column j of M^2 is M applied to column j of M
    for (int j = 0; j < 128; ++j) {
      uint64_t r0 = 0, r1 = 0;
      for (int k = 0; k < 128; ++k) {
        const uint64_t bit = k < 64 ? (cur[2 * j] >> k) & 1 : (cur[2 * j + 1] >> (k - 64)) & 1;
        if (bit) { r0 ^= cur[2 * k]; r1 ^= cur[2 * k + 1]; }
      }
      nxt[2 * j] = r0;
      nxt[2 * j + 1] = r1;
    }
    cur.swap(nxt);
  }
}

int llf_map_index(int cx, int cy) {
  // (cx, cy) in {1,2,4}^2 minus (1,1) and (1,... ) combinations that occur
  if (cx == 2 && cy == 2) return 0;
  if (cx == 4 && cy == 4) return 1;
  if (cx == 1 && cy == 2) return 2;
  if (cx == 2 && cy == 1) return 3;
  if (cx == 1 && cy == 4) return 4;
  if (cx == 4 && cy == 1) return 5;
  if (cx == 2 && cy == 4) return 6;
  if (cx == 4 && cy == 2) return 7;
  return -1;
}

void llf_box_maps(float* out) {
  const int dims[kLlfMaps][2] = {{2, 2}, {4, 4}, {1, 2}, {2, 1},
                                 {1, 4}, {4, 1}, {2, 4}, {4, 2}};
  std::memset(out, 0, sizeof(float) * kLlfMaps * 256);
  for (int m = 0; m < kLlfMaps; ++m) {
    const int cx = dims[m][0], cy = dims[m][1], W = 8 * cx, H = 8 * cy;
    const int n = cx * cy;
    for (int i = 0; i < n; ++i) {
      const int bx = i % cx, by = i / cx;
      for (int j = 0; j < n; ++j) {
        const int u = j % cx, v = j / cx;
        double sx = 0, sy = 0;
        for (int k = 0; k < 8; ++k) {
          sx += std::cos((2 * (8 * bx + k) + 1) * u * kPi / (2.0 * W));
          sy += std::cos((2 * (8 * by + k) + 1) * v * kPi / (2.0 * H));
        }
        out[m * 256 + i * 16 + j] = static_cast<float>((sx / 8) * (sy / 8));
      }
    }
  }
}

void llf_maps(float* out) {
  const int dims[kLlfMaps][2] = {{2, 2}, {4, 4}, {1, 2}, {2, 1},
                                 {1, 4}, {4, 1}, {2, 4}, {4, 2}};
  std::memset(out, 0, sizeof(float) * kLlfMaps * 256);
  for (int m = 0; m < kLlfMaps; ++m) {
    const int cx = dims[m][0], cy = dims[m][1], W = 8 * cx, H = 8 * cy;
    const int n = cx * cy;
    // box-mean map of the unscaled cosine basis: dc[i] = sum_j B[i][j] c~[j]
    std::vector<double> B(n * n);
    for (int i = 0; i < n; ++i) {
      const int bx = i % cx, by = i / cx;
      for (int j = 0; j < n; ++j) {
        const int u = j % cx, v = j / cx;
        double sx = 0, sy = 0;
        for (int k = 0; k < 8; ++k) {
          sx += std::cos((2 * (8 * bx + k) + 1) * u * kPi / (2.0 * W));
          sy += std::cos((2 * (8 * by + k) + 1) * v * kPi / (2.0 * H));
        }
        B[i * n + j] = (sx / 8) * (sy / 8);
      }
    }
    invert(B.data(), n);
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) out[m * 256 + j * 16 + i] = static_cast<float>(B[j * n + i]);
  }
}

void odd_tables(float* out) {
  int off = 0;
  for (int N = 32; N >= 2; N /= 2) {
    for (int n = 0; n < N / 2; ++n)
      for (int j = 0; j < N / 2; ++j)
        out[off + n * (N / 2) + j] =
            static_cast<float>(std::cos((2 * n + 1) * (2 * j + 1) * kPi / (2.0 * N)));
    off += (N / 2) * (N / 2);
  }
}

namespace {
// binary32 bit pattern of Weight(sad, mul) (J.2.4) with mul given as 4 * mul.
uint32_t weight_bits(int64_t sad, int64_t mul4) {
  if (sad > 507) sad = 507;
  int64_t prescaled = sad << 6;
  int64_t p = prescaled * mul4;
  // floor division by 2^18 (arithmetic shift of a signed value)
  int64_t high16 = (p >> 18) + (127 << 7);
  return static_cast<uint32_t>(high16 << 16);
}
}  // namespace

void mul_table4(int32_t* out) {
  std::memset(out, 0, sizeof(int32_t) * 673);
  const int gap = 4;
  int64_t mul = -32768;
  for (int sigma = 16; sigma <= 672; sigma += gap) {
    for (; mul < 0; ++mul) {
      uint32_t b = weight_bits(sigma >> 2, 4 * mul);
      float w;
      std::memcpy(&w, &b, 4);
      if (w > 0.5f) break;
    }
    out[sigma] = static_cast<int32_t>(4 * mul);
  }
  for (int sigma = 16; sigma < 672; sigma += gap) {
    const int32_t step = (out[sigma + gap] - out[sigma]) / gap;  // = mul_step * 4
    for (int i = 1; i < gap; ++i) out[sigma + i] = out[sigma] + i * step;
  }
}

void tc_basis_tables(unsigned char* out) {
  std::memset(out, 0, 6144);
  const int sizes[3] = {8, 16, 32};
  const int offs[3] = {0, 1024, 2048};
  for (int t = 0; t < 3; ++t) {
    const int N = sizes[t], Kp = N < 16 ? 16 : N, sbo = (Kp / 8) * 128;
    unsigned char* hi = out + offs[t];
    unsigned char* lo = hi + Kp * Kp * 2;
    for (int n = 0; n < Kp; ++n) {
      for (int k = 0; k < Kp; ++k) {
        const double v = (n < N && k < N) ? std::cos((2 * n + 1) * k * kPi / (2.0 * N)) : 0.0;
        const __half h = __double2half(v);
        const __half l = __double2half(v - static_cast<double>(__half2float(h)));
        const int off = (n / 8) * sbo + (k / 8) * 128 + (n % 8) * 16 + (k % 8) * 2;
        std::memcpy(hi + off, &h, 2);
        std::memcpy(lo + off, &l, 2);
      }
    }
  }
}

}  // namespace jxlr
