// jxl_recon_run_noalloc: one-call reconstruction that allocates nothing.
//
// Some callers cannot call cudaMalloc: code that runs while another owner
// (a framework's caching allocator, a memory-budgeted service) must account
// for every device byte, or that runs where allocation is not allowed
// because it would synchronise the device.  For them this entry point uses
// device memory that exists for as long as the library is loaded (it
// allocates no device memory; host memory only for the tables it builds on
// its first call per device and for error messages): the
// scratch of the dequantise-and-transform kernel (planar XYB samples and the
// per-block EPF sigma, read back by the filter kernel) lives in a file-scope
// __device__ array of kNoAllocScratchBytes, and the dequantisation matrices
// in another.  Every GPU that loads the library holds both until the
// process exits.
//
// The first call on a device copies the constant tables to it and looks up
// the arrays' device addresses (cudaMemcpyToSymbol / cudaGetSymbolAddress
// with that device current).  That first call should come before any
// stream capture.  Later calls only launch kernels on the caller's stream.
//
// All calls share the arrays and leave their contents behind.  The kernels
// write every scratch element they later read (XYB of every cell, sigma of
// every block), so nothing needs clearing between calls.  Calls whose work
// overlaps on the GPU (different streams, or different host threads on one
// device without ordering) race on the scratch and produce wrong pixels:
// order them on one stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/jxl_recon.h"
#include "internal.h"
#include "kernels.h"

namespace jxlr {
namespace {

constexpr size_t kNoAllocScratchBytes = JXL_RECON_NOALLOC_SCRATCH_BYTES;   // 64 MiB

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
__device__ __align__(256) float g_noalloc_dequant[kDequantFloats];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
bool g_ready[kMaxDevices];
unsigned char* g_scratch_ptr[kMaxDevices];
float* g_dequant_ptr[kMaxDevices];
jxlr_status noalloc_fail(jxlr_status s, const std::string& m) {
  set_last_error(m);   // read back with jxl_recon_last_error(NULL)
  return s;
}

// Once per device, with that device current.
jxlr_status setup_device(int dev) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (g_ready[dev]) return JXLR_OK;
  std::vector<float> raw(kDequantFloats), scaled(kDequantFloats);
  if (!default_dequant(raw.data())) return noalloc_fail(JXLR_EINVAL, "default matrices ill-formed");
  prescale_dequant(raw.data(), scaled.data());
  std::vector<float> llf(kLlfMaps * 256), box(kLlfMaps * 256), odd(kOddFloats), afv(256);
  std::vector<int32_t> mul4(673);
  llf_maps(llf.data());
  llf_box_maps(box.data());
  odd_tables(odd.data());
  mul_table4(mul4.data());
  for (int j = 0; j < 16; ++j)
    for (int i = 0; i < 16; ++i) afv[j * 16 + i] = static_cast<float>(kAfvBasis[j][i]);
  if (!upload_constants(llf.data(), box.data(), odd.data(), mul4.data(), afv.data()))
    return noalloc_fail(JXLR_ECUDA, "noalloc setup: constant upload failed");
  cudaError_t e = cudaMemcpyToSymbol(g_noalloc_dequant, scaled.data(),
                                     sizeof(float) * kDequantFloats);
  if (e != cudaSuccess)
    return noalloc_fail(JXLR_ECUDA, std::string("noalloc setup: ") + cudaGetErrorString(e));
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess)
    return noalloc_fail(JXLR_ECUDA, std::string("noalloc scratch address: ") + cudaGetErrorString(e));
  g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  e = cudaGetSymbolAddress(&p, g_noalloc_dequant);
  if (e != cudaSuccess)
    return noalloc_fail(JXLR_ECUDA, std::string("noalloc table address: ") + cudaGetErrorString(e));
  g_dequant_ptr[dev] = static_cast<float*>(p);
  g_ready[dev] = true;
  return JXLR_OK;
}

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace
}  // namespace jxlr

using namespace jxlr;

extern "C" jxlr_status jxl_recon_run_noalloc(const jxl_recon_coeffs* co, const uint8_t* vmap,
                                             const float* qf, const jxl_recon_cfl* cfl,
                                             const jxl_recon_filter_params* fp,
                                             const jxl_recon_output* out, void* cuda_stream) {
  if (!co || !vmap || !qf || !cfl || !cfl->k || !fp || !out)
    return noalloc_fail(JXLR_EINVAL, "run_noalloc: null argument");
  if (!co->on_device || !out->on_device)
    return noalloc_fail(JXLR_EINVAL, "run_noalloc: inputs and output must be device buffers");
  if (fp->dequant)
    return noalloc_fail(JXLR_EINVAL, "run_noalloc: custom dequant matrices are not supported");
  const int xs = static_cast<int>(co->xsize), ys = static_cast<int>(co->ysize);
  if (xs <= 0 || ys <= 0 || xs > 65536 || ys > 65536)
    return noalloc_fail(JXLR_EINVAL, "run_noalloc: image size out of [1, 65536]");
  const int wp = (xs + 7) & ~7, hp = (ys + 7) & ~7, bw = wp / 8, bh = hp / 8;
  const int tw = (wp + 63) / 64;
  const bool filters = fp->epf || fp->gab;
  const size_t xyb_bytes = up256(sizeof(float) * 3 * size_t(wp) * hp);
  const size_t sig_bytes = up256(sizeof(int16_t) * size_t(bw) * bh);
  if (filters && xyb_bytes + sig_bytes > kNoAllocScratchBytes)
    return noalloc_fail(JXLR_EINVAL,
                        "run_noalloc: padded image needs " + std::to_string(xyb_bytes + sig_bytes) +
                            " scratch bytes, above the fixed " +
                            std::to_string(kNoAllocScratchBytes));
  if (co->row_stride_elems < size_t(wp) || co->row_stride_elems % 8)
    return noalloc_fail(JXLR_EINVAL, "run_noalloc: coefficient row stride");
  for (int c = 0; c < 3; ++c)
    if (!co->plane[c] || (reinterpret_cast<uintptr_t>(co->plane[c]) & 15))
      return noalloc_fail(JXLR_EINVAL, "run_noalloc: coefficient planes must be 16-byte aligned");
  if (out->dtype < 0 || out->dtype > 3 || !out->data)
    return noalloc_fail(JXLR_EINVAL, "run_noalloc: bad output");
  const size_t px_bytes = out->dtype == 1 ? 6 : out->dtype == 2 ? 3 : 12;
  if (out->row_stride_bytes < px_bytes * xs)
    return noalloc_fail(JXLR_EINVAL, "run_noalloc: output stride too small");
  if (fp->epf && !fp->sharpness)
    return noalloc_fail(JXLR_EINVAL, "run_noalloc: EPF needs the sharpness map");
  if (fp->dc_smooth || fp->lf_predict || (fp->epf && fp->qco) || fp->noise)
    return noalloc_fail(JXLR_EINVAL, "run_noalloc: DC smoothing, AC prediction and the quantization constraint run on the submit path only");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(JXLR_ECUDA, "run_noalloc: no current device");
  jxlr_status st = setup_device(dev);
  if (st != JXLR_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

  ReconArgs ra;
  std::memset(&ra, 0, sizeof(ra));
  for (int c = 0; c < 3; ++c) ra.coef[c] = co->plane[c];
  ra.cstride = co->row_stride_elems;
  ra.vmap = vmap;
  ra.acmul = qf;
  ra.cfl = cfl->k;
  ra.sharp = fp->sharpness;
  ra.dequant = g_dequant_ptr[dev];
  ra.xs = xs; ra.ys = ys; ra.wp = wp; ra.hp = hp; ra.bw = bw; ra.bh = bh; ra.tw = tw;
  for (int c = 0; c < 3; ++c) {
    ra.m_dc[c] = fp->m_dc[c];
    ra.one_minus_bias[c] = one_minus_bias(c);
  }
  ra.kx_dc = cfl->kx_dc;
  ra.kb_dc = cfl->kb_dc;
  // the same parameter derivations as the context path
  ra.sp = sigma_params(*fp);
  ra.cp = color_params(*fp);
  OutParams op;
  op.data = out->data;
  op.stride = out->row_stride_bytes;
  op.dtype = out->dtype;

  if (filters) {
    float* xyb = reinterpret_cast<float*>(g_scratch_ptr[dev]);
    int16_t* sig = fp->epf ? reinterpret_cast<int16_t*>(g_scratch_ptr[dev] + xyb_bytes) : nullptr;
    ra.write_xyb = 1;
    ra.xyb = xyb;
    ra.sigma = sig;
    launch_recon(ra, s);
    FilterArgs fa = filter_args(*fp);
    fa.xyb = xyb;
    fa.rstride = wp;
    fa.pstride = size_t(wp) * hp;
    fa.xs = xs; fa.ys = ys; fa.bw = bw;
    fa.sigma = sig;
    fa.out = op;
    // With the EPF: the single-launch J.2 + J.4 + L.2 kernel (no buffer for
    // an intermediate image).  Gaborish alone: the form that loads its tiles
    // with ordinary loads, which has no bounded wait whose expiry this call
    // (which returns before the kernels run) could not report.
    if (fp->epf) launch_filter(fa, s);
    else launch_filter_plain(fa, s);
  } else {
    ra.write_xyb = 0;
    ra.out = op;
    launch_recon(ra, s);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return noalloc_fail(JXLR_ECUDA, std::string("run_noalloc launch: ") + cudaGetErrorString(e));
  return JXLR_OK;
}
