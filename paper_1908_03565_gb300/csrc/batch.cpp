// Multi-image batches: one launch per kernel kind for many uneven images,
// captured once in a CUDA graph and replayed.
//
// Every image keeps its own parameter block (sizes, pointers, filters,
// output encoding) in device memory; the multi-image kernels map their work
// items (32x32 cells for the transforms, filter tiles) to (image, cell) by a
// prefix array.  With the EPF, the transform kernel lists each image's 8x8
// blocks with sigma >= 16 (and copies the others to its J.2 buffer), the
// J.2 kernel's persistent warps take the images' listed blocks round robin,
// and Gaborish + colour run on the J.2 buffers with the other images'
// filter tiles.  With JXLR_BATCH_AUTOTUNE the grids of the three kernel kinds
// and the form of the Gaborish / colour kernel (TMA tiles or ordinary
// loads) are chosen by timing candidates on the batch itself, all of which
// compute the same bits, and remembered per batch class (images, cells,
// images with the EPF, filter tiles, output-type mix; in this process, and
// in the file named by $JXLR_AUTOTUNE_CACHE if set).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/jxl_recon.h"
#include "internal.h"
#include "kernels.h"

using namespace jxlr;

struct jxl_recon_batch {
  jxl_recon_ctx* ctx = nullptr;
  int device = 0;
  uint32_t n = 0;
  uint64_t pixels = 0;
  char* dmem = nullptr;
  ReconArgs* d_rargs = nullptr;
  int* d_ritem = nullptr;          // per transform work item: (image, cell in it)
  int rtotal = 0;
  FilterArgs* d_eargs = nullptr;   // J.2 of the images with the EPF
  unsigned* d_counts = nullptr;    // their listed-block counts, then the J.2 group counter
                                   // (ne + 1 words, zeroed per launch)
  int ne = 0, etotal = 0;
  bool clamp = false;
  FilterArgs* d_fargs = nullptr;   // Gaborish / colour of every filtered image
  int* d_fprefix = nullptr;
  int nf = 0, ftotal = 0;
  void* d_maps = nullptr;          // their tensor maps (TMA form of the filter), or null
  unsigned* d_err = nullptr;       // bit 8: a bounded tile-load wait of the filter expired
  bool use_tma = false;            // the filter runs in its TMA form (d_maps set)
  int grid[3] = {0, 0, 0};         // recon, epf, filter
  float kind_ms[3] = {0, 0, 0};    // the tuned kernels' times (autotune), ms
  uint32_t mix = 0;                // output types: 8 bits per count of f32 / f16 / u8 (capped)
  int autotuned = 0;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int kernels = 0;
};

namespace {

size_t up(size_t v, size_t a) { return (v + a - 1) / a * a; }

jxlr_status bfail(jxlr_status s, const std::string& m) {
  set_last_error(m);
  return s;
}

void enqueue(const jxl_recon_batch* b, const int* grid, cudaStream_t s) {
  if (b->ne) cudaMemsetAsync(b->d_counts, 0, sizeof(unsigned) * (b->ne + 1), s);
  if (b->rtotal) launch_recon_batch(b->d_rargs, b->d_ritem, b->rtotal, grid[0], s);
  if (b->ne)
    launch_epf_work_batch(b->d_eargs, b->d_counts, b->ne, b->clamp, grid[1], b->d_counts + b->ne,
                          s);
  if (b->ftotal) {
    if (b->use_tma)
      launch_filter_batch_tma(b->d_fargs, b->d_fprefix, b->d_maps, b->nf, b->ftotal, grid[2],
                              b->d_err, s);
    else
      launch_filter_batch(b->d_fargs, b->d_fprefix, b->nf, b->ftotal, grid[2], s);
  }
}

// A batch class: images, transform cells, images with the EPF, filter
// tiles, output-type mix.  The tuned choice: grids of the three kernel kinds
// and the filter's form (1: TMA tiles, 0: ordinary loads).
using Key = std::tuple<uint32_t, int, int, int, uint32_t>;
struct Choice {
  int grid[3];
  int tma;
  float ms[3];
};
std::mutex g_tune_mu;
std::map<Key, Choice> g_tuned;

bool tuned_lookup(const Key& k, Choice* c) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tuned.find(k);
  if (it == g_tuned.end()) {
    const char* path = std::getenv("JXLR_AUTOTUNE_CACHE");
    if (!path) return false;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
      std::istringstream in(line);
      uint32_t n, mix;
      int a, bb, cc;
      Choice ch;
      if (in >> n >> a >> bb >> cc >> mix >> ch.grid[0] >> ch.grid[1] >> ch.grid[2] >> ch.tma >>
          ch.ms[0] >> ch.ms[1] >> ch.ms[2])
        g_tuned[Key(n, a, bb, cc, mix)] = ch;
    }
    it = g_tuned.find(k);
    if (it == g_tuned.end()) return false;
  }
  *c = it->second;
  return true;
}

void tuned_store(const Key& k, const Choice& c) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tuned[k] = c;
  if (const char* path = std::getenv("JXLR_AUTOTUNE_CACHE")) {
    std::ofstream f(path, std::ios::app);
    f << std::get<0>(k) << ' ' << std::get<1>(k) << ' ' << std::get<2>(k) << ' '
      << std::get<3>(k) << ' ' << std::get<4>(k) << ' ' << c.grid[0] << ' ' << c.grid[1] << ' '
      << c.grid[2] << ' ' << c.tma << ' ' << c.ms[0] << ' ' << c.ms[1] << ' ' << c.ms[2] << '\n';
  }
}

// One kernel kind of the batch alone (k: 0 transform, 1 J.2, 2 Gaborish /
// colour in the form tma) on grid g, on the batch's stream.  The transform
// appends to the J.2 lists, so they restart empty; J.2 reads the lists the
// last transform run left.
void launch_kind(jxl_recon_batch* b, int k, int g, bool tma) {
  if (k == 0) {
    if (b->ne) cudaMemsetAsync(b->d_counts, 0, sizeof(unsigned) * (b->ne + 1), b->cap);
    launch_recon_batch(b->d_rargs, b->d_ritem, b->rtotal, g, b->cap);
  } else if (k == 1) {
    cudaMemsetAsync(b->d_counts + b->ne, 0, sizeof(unsigned), b->cap);
    launch_epf_work_batch(b->d_eargs, b->d_counts, b->ne, b->clamp, g, b->d_counts + b->ne, b->cap);
  } else if (tma) {
    launch_filter_batch_tma(b->d_fargs, b->d_fprefix, b->d_maps, b->nf, b->ftotal, g, b->d_err,
                            b->cap);
  } else {
    launch_filter_batch(b->d_fargs, b->d_fprefix, b->nf, b->ftotal, g, b->cap);
  }
}

// Times the candidate forms and grids of each kernel kind on the batch
// itself and keeps the fastest (median of 3 after a warm-up).  Every
// candidate computes the same bits: the grids only change which CTA takes
// which work item, the two filter forms load the same tile with TMA or with
// ordinary loads.  Candidates: transform one CTA per cell or 1, 2, 4 x the
// resident CTAs; J.2 (persistent warps) 1/2, 3/4 or all of the resident
// warps; Gaborish / colour in the TMA form on all or half of its resident
// CTAs, or with ordinary loads on one CTA per tile or 1, 2 x the resident
// CTAs.
jxlr_status autotune(jxl_recon_batch* b, bool tma_allowed) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto time_it = [&](int k, int g, bool tma) {
    std::vector<float> t;
    for (int rep = 0; rep < 4; ++rep) {
      cudaEventRecord(e0, b->cap);
      launch_kind(b, k, g, tma);
      cudaEventRecord(e1, b->cap);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep) t.push_back(ms);
    }
    std::sort(t.begin(), t.end());
    return t[1];
  };
  for (int k = 0; k < 3; ++k) {
    struct Cand {
      int g;
      bool tma;
    };
    std::vector<Cand> cand;
    if (k == 0 && b->rtotal) {
      const int res = sms * batch_blocks_per_sm(0);
      cand.push_back({b->rtotal, false});
      for (int f : {1, 2, 4})
        if (f * res < b->rtotal) cand.push_back({f * res, false});
    } else if (k == 1 && b->ne) {
      const int res = sms * batch_blocks_per_sm(1);
      for (int num : {2, 3, 4}) cand.push_back({std::max(1, res * num / 4), false});
    } else if (k == 2 && b->ftotal) {
      if (tma_allowed) {
        const int res = sms * batch_blocks_per_sm(3);
        cand.push_back({res, true});
        cand.push_back({std::max(1, res / 2), true});
      }
      const int res = sms * batch_blocks_per_sm(2);
      cand.push_back({b->ftotal, false});
      for (int f : {1, 2})
        if (f * res < b->ftotal) cand.push_back({f * res, false});
    }
    if (cand.empty()) continue;
    if (k == 1) launch_kind(b, 0, b->grid[0], false);   // the lists J.2 reads
    float best = 1e30f;
    for (const Cand& c : cand) {
      const float ms = time_it(k, c.g, c.tma);
      if (ms < best) {
        best = ms;
        b->grid[k] = c.g;
        if (k == 2) b->use_tma = c.tma;
      }
    }
    b->kind_ms[k] = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? JXLR_OK : bfail(JXLR_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
}

}  // namespace

extern "C" jxlr_status jxl_recon_batch_destroy(jxl_recon_batch* b) {
  if (!b) return JXLR_OK;
  cudaSetDevice(b->device);
  if (b->cap) cudaStreamSynchronize(b->cap);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->dmem) cudaFree(b->dmem);
  delete b;
  return JXLR_OK;
}

extern "C" jxlr_status jxl_recon_batch_create(jxl_recon_ctx* ctx, const jxl_recon_request* reqs,
                                              size_t n, int flags, jxl_recon_batch** out) {
  if (!ctx || !reqs || !out || n == 0 || n > (1u << 20))
    return bfail(JXLR_EINVAL, "batch_create: bad arguments");
  if (ctx_precision(ctx) != JXLR_PREC_FP32)
    return bfail(JXLR_EINVAL, "batch_create: batches run the FP32 path only (a context created "
                              "with JXLR_PREC_FP32)");
  const int dev = ctx_device(ctx);
  if (cudaSetDevice(dev) != cudaSuccess) return bfail(JXLR_ECUDA, "batch_create: set device");
  std::vector<ReconArgs> ra(n);
  std::vector<FilterArgs> ea, fa;
  std::vector<int> rpre(1, 0), fpre(1, 0);
  std::vector<size_t> scratch_off(n, 0), sig_off(n, 0), eo_off(n, 0), list_off(n, 0);
  std::vector<int> eimg, fimg;
  size_t scratch = 0;
  uint64_t pixels = 0;
  for (size_t i = 0; i < n; ++i) {
    const jxl_recon_request& r = reqs[i];
    const jxl_recon_coeffs* co = r.coeffs;
    const jxl_recon_filter_params* fp = r.filter_params;
    const jxl_recon_output* o = r.out;
    if (!co || !fp || !o || !r.varblock_map || !r.quant_field || !r.cfl_map || !r.cfl_map->k)
      return bfail(JXLR_EINVAL, "batch_create: null field in request " + std::to_string(i));
    if (!co->on_device || !o->on_device || fp->dequant)
      return bfail(JXLR_EINVAL, "batch_create: requests must be device-resident with default matrices");
    const int xs = static_cast<int>(co->xsize), ys = static_cast<int>(co->ysize);
    if (xs <= 0 || ys <= 0 || xs > 65536 || ys > 65536)
      return bfail(JXLR_EINVAL, "batch_create: image size");
    const int wp = (xs + 7) & ~7, hp = (ys + 7) & ~7, bw = wp / 8, bh = hp / 8;
    if (co->row_stride_elems < size_t(wp) || co->row_stride_elems % 8)
      return bfail(JXLR_EINVAL, "batch_create: coefficient row stride");
    for (int c = 0; c < 3; ++c)
      if (!co->plane[c] || (reinterpret_cast<uintptr_t>(co->plane[c]) & 15))
        return bfail(JXLR_EINVAL, "batch_create: coefficient planes must be 16-byte aligned");
    const size_t px_bytes = o->dtype == 1 ? 6 : o->dtype == 2 ? 3 : 12;
    if (o->dtype < 0 || o->dtype > 3 || !o->data || o->row_stride_bytes < px_bytes * xs)
      return bfail(JXLR_EINVAL, "batch_create: bad output");
    if (fp->epf && !fp->sharpness) return bfail(JXLR_EINVAL, "batch_create: EPF needs sharpness");
    if (fp->dc_smooth || fp->lf_predict || (fp->epf && fp->qco) || fp->noise)
      return bfail(JXLR_EINVAL, "batch_create: DC smoothing, AC prediction and the quantization constraint run on the submit path only (so does noise)");
    pixels += uint64_t(xs) * ys;
    ReconArgs& a = ra[i];
    std::memset(&a, 0, sizeof(a));
    for (int c = 0; c < 3; ++c) a.coef[c] = co->plane[c];
    a.cstride = co->row_stride_elems;
    a.vmap = r.varblock_map;
    a.acmul = r.quant_field;
    a.cfl = r.cfl_map->k;
    a.sharp = fp->sharpness;
    a.dequant = ctx_default_dequant(ctx);
    a.xs = xs; a.ys = ys; a.wp = wp; a.hp = hp; a.bw = bw; a.bh = bh; a.tw = (wp + 63) / 64;
    for (int c = 0; c < 3; ++c) {
      a.m_dc[c] = fp->m_dc[c];
      a.one_minus_bias[c] = one_minus_bias(c);
    }
    a.kx_dc = r.cfl_map->kx_dc;
    a.kb_dc = r.cfl_map->kb_dc;
    a.sp = sigma_params(*fp);
    a.cp = color_params(*fp);
    OutParams op;
    op.data = o->data;
    op.stride = o->row_stride_bytes;
    op.dtype = o->dtype;
    rpre.push_back(rpre.back() + ((wp + 31) / 32) * ((hp + 31) / 32));
    if (fp->epf || fp->gab) {
      a.write_xyb = 1;
      scratch = up(scratch, 256);
      scratch_off[i] = scratch;
      scratch += sizeof(float) * 3 * size_t(wp) * hp;
      if (fp->epf) {
        scratch = up(scratch, 256);
        sig_off[i] = scratch;
        scratch += sizeof(int16_t) * size_t(bw) * bh;
        scratch = up(scratch, 256);
        eo_off[i] = scratch;                              // J.2 output
        scratch += sizeof(float) * 3 * size_t(wp) * hp;
        scratch = up(scratch, 256);
        list_off[i] = scratch;                            // listed blocks
        scratch += sizeof(int) * size_t(bw) * bh;
      }
      FilterArgs f = filter_args(*fp);
      f.rstride = wp;
      f.pstride = size_t(wp) * hp;
      f.xs = xs; f.ys = ys; f.bw = bw;
      f.out = op;
      if (fp->epf) {
        f.ors = wp;
        f.ops = size_t(wp) * hp;
        ea.push_back(f);
        eimg.push_back(static_cast<int>(i));
      }
      FilterArgs g = f;   // J.4 / L.2 (on the J.2 output with the EPF)
      g.epf = 0;
      fa.push_back(g);
      fimg.push_back(static_cast<int>(i));
      fpre.push_back(fpre.back() + filter_tiles(g));
    } else {
      a.write_xyb = 0;
      a.out = op;
    }
  }
  auto* b = new jxl_recon_batch();
  b->ctx = ctx;
  b->device = dev;
  b->n = static_cast<uint32_t>(n);
  b->pixels = pixels;
  b->ne = static_cast<int>(ea.size());
  b->nf = static_cast<int>(fa.size());
  b->rtotal = rpre.back();
  b->etotal = b->ne;
  b->ftotal = fpre.back();
  // one device allocation: parameter blocks, prefixes, statuses, scratch
  size_t off = 0;
  auto take = [&](size_t bytes) { off = up(off, 256); size_t o = off; off += bytes; return o; };
  // per transform work item: its image and its cell within the image
  std::vector<int> ritem(2 * static_cast<size_t>(rpre.back()));
  for (size_t i = 0; i < n; ++i)
    for (int w = rpre[i]; w < rpre[i + 1]; ++w) {
      ritem[2 * static_cast<size_t>(w)] = static_cast<int>(i);
      ritem[2 * static_cast<size_t>(w) + 1] = w - rpre[i];
    }
  const size_t o_r = take(sizeof(ReconArgs) * n), o_rp = take(sizeof(int) * ritem.size());
  const size_t o_e = take(sizeof(FilterArgs) * ea.size()), o_ec = take(sizeof(unsigned) * (ea.size() + 1));
  const size_t o_f = take(sizeof(FilterArgs) * fa.size()), o_fp = take(sizeof(int) * fpre.size());
  const size_t o_st = take(sizeof(unsigned) * 4 * n);
  // one tensor map per filtered image when every one of them allows TMA
  struct alignas(64) Map { unsigned char b[kTensorMapBytes]; };
  std::vector<Map> maps(fa.size());
  bool tma = !fa.empty() && !(flags & JXLR_BATCH_PLAIN_LOADS);
  const size_t o_tm = take(sizeof(Map) * fa.size()), o_er = take(sizeof(unsigned));
  const size_t o_sc = take(scratch);
  cudaError_t e = cudaMalloc(&b->dmem, up(off, 256));
  if (e != cudaSuccess) {
    cudaGetLastError();
    jxl_recon_batch_destroy(b);
    return bfail(JXLR_ENOMEM, "batch_create: device allocation failed");
  }
  char* base = b->dmem;
  b->d_counts = reinterpret_cast<unsigned*>(base + o_ec);
  std::vector<float*> eo(n, nullptr);
  for (size_t i = 0; i < n; ++i) {
    if (ra[i].write_xyb) {
      ra[i].xyb = reinterpret_cast<float*>(base + o_sc + scratch_off[i]);
      ra[i].sigma = reqs[i].filter_params->epf
                        ? reinterpret_cast<int16_t*>(base + o_sc + sig_off[i]) : nullptr;
    }
  }
  for (size_t j = 0; j < ea.size(); ++j) {
    ReconArgs& r = ra[eimg[j]];
    eo[eimg[j]] = reinterpret_cast<float*>(base + o_sc + eo_off[eimg[j]]);
    r.epf.list = reinterpret_cast<int*>(base + o_sc + list_off[eimg[j]]);
    r.epf.count = b->d_counts + j;
    r.epf.pass = eo[eimg[j]];
    r.epf.prs = size_t(r.wp);
    r.epf.pps = size_t(r.wp) * r.hp;
    ea[j].xyb = r.xyb;
    ea[j].sigma = r.sigma;
    ea[j].epf_out = eo[eimg[j]];
    ea[j].epf_list = r.epf.list;
    ea[j].epf_count = r.epf.count;
    b->clamp = b->clamp || filter_needs_clamp(ea[j]);
  }
  for (size_t j = 0; j < fa.size(); ++j) {
    const int i = fimg[j];
    fa[j].xyb = eo[i] ? eo[i] : ra[i].xyb;
    fa[j].sigma = nullptr;
    tma = tma && make_filter_tensor_map(fa[j], &maps[j]);
  }
  if (tma) {
    b->d_maps = base + o_tm;
    b->d_err = reinterpret_cast<unsigned*>(base + o_er);
    b->use_tma = true;
  }
  b->d_rargs = reinterpret_cast<ReconArgs*>(base + o_r);
  b->d_ritem = reinterpret_cast<int*>(base + o_rp);
  b->d_eargs = reinterpret_cast<FilterArgs*>(base + o_e);
  b->d_fargs = reinterpret_cast<FilterArgs*>(base + o_f);
  b->d_fprefix = reinterpret_cast<int*>(base + o_fp);
  unsigned* d_status = reinterpret_cast<unsigned*>(base + o_st);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  auto h2d = [&](void* d, const void* h, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, b->cap);
  };
  h2d(b->d_rargs, ra.data(), sizeof(ReconArgs) * n);
  h2d(b->d_ritem, ritem.data(), sizeof(int) * ritem.size());
  h2d(b->d_eargs, ea.data(), sizeof(FilterArgs) * ea.size());
  h2d(b->d_fargs, fa.data(), sizeof(FilterArgs) * fa.size());
  h2d(b->d_fprefix, fpre.data(), sizeof(int) * fpre.size());
  if (b->d_maps) h2d(b->d_maps, maps.data(), sizeof(Map) * maps.size());
  if (b->d_err && e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, sizeof(unsigned), b->cap);
  // C.5.4 validation of every map, once, at creation
  if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(unsigned) * 4 * n, b->cap);
  for (size_t i = 0; i < n && e == cudaSuccess; ++i)
    launch_validate(reqs[i].varblock_map, ra[i].bw, ra[i].bh, d_status + 4 * i, b->cap);
  std::vector<unsigned> st(4 * n);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(st.data(), d_status, sizeof(unsigned) * 4 * n, cudaMemcpyDeviceToHost, b->cap);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->cap);
  if (e != cudaSuccess) {
    jxl_recon_batch_destroy(b);
    return bfail(JXLR_ECUDA, std::string("batch_create: ") + cudaGetErrorString(e));
  }
  for (size_t i = 0; i < n; ++i)
    if (st[4 * i] != 0) {
      jxl_recon_batch_destroy(b);
      return bfail(JXLR_EINVAL, "batch_create: DctSelect map of request " + std::to_string(i) +
                                    " is ill-formed");
    }
  ctx_count_launches(ctx, static_cast<int>(n));
  // grids and filter form: cached tuning, fresh tuning, or one CTA per work
  // item (the J.2 kernel and the TMA form of the filter on their resident grids)
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->grid[0] = b->rtotal;
  b->grid[1] = b->ne ? sms * batch_blocks_per_sm(1) : 0;
  b->grid[2] = b->use_tma ? sms * batch_blocks_per_sm(3) : b->ftotal;
  for (size_t i = 0; i < n; ++i) {
    const int dt = reqs[i].out->dtype == JXLR_OUT_U8_SRGB ? 0 : reqs[i].out->dtype == JXLR_OUT_F16_LINEAR ? 8 : 16;
    if (((b->mix >> dt) & 0xFF) < 0xFF) b->mix += 1u << dt;
  }
  const Key key(b->n, b->rtotal, b->etotal, b->ftotal, b->mix);
  Choice ch;
  if (tuned_lookup(key, &ch) && (!ch.tma || b->d_maps)) {
    for (int k = 0; k < 3; ++k) {
      b->grid[k] = ch.grid[k];
      b->kind_ms[k] = ch.ms[k];
    }
    b->use_tma = ch.tma != 0;
    b->autotuned = 2;
  } else if (flags & JXLR_BATCH_AUTOTUNE) {
    jxlr_status ts = autotune(b, b->d_maps != nullptr);
    if (ts != JXLR_OK) {
      jxl_recon_batch_destroy(b);
      return ts;
    }
    for (int k = 0; k < 3; ++k) {
      ch.grid[k] = b->grid[k];
      ch.ms[k] = b->kind_ms[k];
    }
    ch.tma = b->use_tma;
    tuned_store(key, ch);
    b->autotuned = 1;
  }
  for (int k = 0; k < 3; ++k) b->grid[k] = std::max(1, b->grid[k]);
  // capture the launches once
  e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    enqueue(b, b->grid, b->cap);
    e = cudaStreamEndCapture(b->cap, &b->graph);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) {
    jxl_recon_batch_destroy(b);
    return bfail(JXLR_ECUDA, std::string("batch graph: ") + cudaGetErrorString(e));
  }
  b->kernels = (b->rtotal > 0) + (b->ne > 0) + (b->ftotal > 0);
  *out = b;
  return JXLR_OK;
}

extern "C" jxlr_status jxl_recon_batch_launch(jxl_recon_batch* b, void* cuda_stream) {
  if (!b) return bfail(JXLR_EINVAL, "batch_launch: null batch");
  if (cudaSetDevice(b->device) != cudaSuccess) return bfail(JXLR_ECUDA, "batch_launch: set device");
  cudaError_t e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return bfail(JXLR_ECUDA, std::string("batch_launch: ") + cudaGetErrorString(e));
  ctx_count_launches(b->ctx, b->kernels);
  return JXLR_OK;
}

extern "C" jxlr_status jxl_recon_batch_query(const jxl_recon_batch* b, jxl_recon_batch_info* info) {
  if (!b || !info) return bfail(JXLR_EINVAL, "batch_query: null argument");
  info->images = b->n;
  info->pixels = b->pixels;
  info->recon_items = b->rtotal;
  info->epf_items = b->etotal;
  info->filter_items = b->ftotal;
  info->recon_grid = b->grid[0];
  info->epf_grid = b->grid[1];
  info->filter_grid = b->grid[2];
  info->kernels_per_launch = b->kernels;
  info->autotuned = b->autotuned;
  info->filter_tma = b->use_tma;
  for (int k = 0; k < 3; ++k) info->kind_ms[k] = b->kind_ms[k];
  info->mix = b->mix;
  return JXLR_OK;
}

extern "C" jxlr_status jxl_recon_batch_status(const jxl_recon_batch* b, uint32_t* flags) {
  if (!b || !flags) return bfail(JXLR_EINVAL, "batch_status: null argument");
  *flags = 0;
  if (!b->d_err) return JXLR_OK;
  if (cudaSetDevice(b->device) != cudaSuccess ||
      cudaMemcpy(flags, b->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess)
    return bfail(JXLR_ECUDA, "batch_status: read failed");
  return JXLR_OK;
}
