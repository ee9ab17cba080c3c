// C ABI of libjxlrecon: contexts, slots (one stream + scratch arena each),
// admission under an HBM cap, request tickets.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/jxl_recon.h"
#include "internal.h"
#include "kernels.h"
#include "jpeg1.h"
#include "lf.h"
#include "noise.h"

using namespace jxlr;

namespace {

thread_local std::string g_err;

jxlr_status fail(jxlr_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

jxlr_status cuda_fail(cudaError_t e, const char* what) {
  return fail(JXLR_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

using Clock = std::chrono::steady_clock;

}  // namespace

void jxlr::set_last_error(const std::string& msg) { g_err = msg; }

namespace {

constexpr int kMaxPrio = 8;   // stream priority levels a slot keeps a stream for

struct Slot {
  cudaStream_t stream = nullptr;   // the stream of the current request
  bool own_stream = true;
  // the slot's streams, one per priority level from the lowest (0) up; a
  // request runs on the one of its size class
  cudaStream_t pstream[kMaxPrio] = {};
  int nprio = 0;
  cudaEvent_t done = nullptr;
  // timing marks: start, staged, validated, recon, end, before J.2, after J.2
  cudaEvent_t ev[7] = {};
  bool epf_marked = false;    // marks 5 and 6 were recorded for this request
  char* arena = nullptr;
  size_t arena_bytes = 0;
  unsigned* h_status = nullptr;   // pinned: device status copied back here
  bool busy = false;
  bool timed = false;
  bool check_status = false;
  uint64_t ticket = 0;
  Clock::time_point t_submit;
};

struct Timing {
  float ms[4];
  float epf_ms = 0.f;
  unsigned epf_blocks = 0;
};

// Words of the per-request device status block: [0] validation flags,
// [1] [2] validation counters, [3] a bounded device wait expired (4: the
// tensor-core completion, 8: a filter tile load), [4] blocks the J.2 kernel
// filtered, [5] the J.2 kernel's group counter (its warps claim work there).
constexpr int kStatusWords = 8;

}  // namespace

struct jxl_recon_ctx {
  int device = 0;
  size_t cap = 0;
  bool timing = false;
  std::vector<Slot> slots;
  float* d_dequant = nullptr;        // prescaled default matrices
  int precision = JXLR_PREC_FP32;
  int recon_variant = kReconGrid;    // form of the FP32 transform kernel
  unsigned char* d_tcb = nullptr;    // tensor-core basis tables
  std::mutex mu;
  std::atomic<uint64_t> next_ticket{1};
  std::atomic<uint64_t> launches{0};
  size_t bytes = 0;                  // sum of slot arenas
  std::unordered_map<uint64_t, Timing> timings;
};

namespace jxlr {
const float* ctx_default_dequant(const jxl_recon_ctx* c) { return c->d_dequant; }
int ctx_idle_slots(jxl_recon_ctx* c) {
  std::lock_guard<std::mutex> lock(c->mu);
  int n = 0;
  for (const auto& s : c->slots) n += !s.busy;
  return n;
}
int ctx_device(const jxl_recon_ctx* c) { return c->device; }
int ctx_precision(const jxl_recon_ctx* c) { return c->precision; }
void ctx_count_launches(jxl_recon_ctx* c, int n) { c->launches += n; }
}  // namespace jxlr

extern "C" {

void jxl_recon_filter_defaults(jxl_recon_filter_params* p) {
  std::memset(p, 0, sizeof(*p));
  p->gab = 0;
  for (int c = 0; c < 3; ++c) {
    p->gab_w1[c] = 0.115169525f;
    p->gab_w2[c] = 0.061248592f;
  }
  p->epf = 0;
  p->epf_weight_min = 0.3f;
  p->epf_scale[0] = 899.676941f;
  p->epf_scale[1] = 111.965157f;
  p->epf_scale[2] = 45.275791f;
  for (int i = 0; i < 8; ++i) p->epf_sharp_lut[i] = static_cast<float>(i / 7.0);
  p->epf_range_max = 70.0f;
  p->epf_range_mul = 12.6f;
  p->epf_quant_mul = 20.0f;
  p->epf_sigma_max = 170;
  p->sharpness = nullptr;
  const double r2 = 64.0 * std::sqrt(2.0);
  p->m_dc[0] = static_cast<float>(0.02 / r2);
  p->m_dc[1] = static_cast<float>(0.2 / r2);
  p->m_dc[2] = static_cast<float>(0.2 / r2);
  const float m[9] = {2542.56835937500000f, -2326.53173828125000f, 44.17734527587891f,
                      -698.04852294921875f, 1012.71777343750000f, -76.22974395751953f,
                      -827.36480712890625f, 709.83502197265625f, 451.38488769531250f};
  std::memcpy(p->inv_opsin, m, sizeof(m));
  p->opsin_bias[0] = -0.00100549f;
  p->opsin_bias[1] = -0.00100549f;
  p->opsin_bias[2] = -0.00094081f;
  p->target_nits_div50 = 5;
  p->dequant = nullptr;
  p->qco = 0;
  p->qco_interval_mul = 0.5f;
}

const char* jxl_recon_last_error(const jxl_recon_ctx*) { return g_err.c_str(); }

uint64_t jxl_recon_launch_count(const jxl_recon_ctx* ctx) { return ctx ? ctx->launches.load() : 0; }

size_t jxl_recon_device_bytes(const jxl_recon_ctx* ctx) { return ctx ? ctx->bytes : 0; }

jxlr_status jxl_recon_create(const jxl_recon_config* cfg, jxl_recon_ctx** out) {
  if (!cfg || !out) return fail(JXLR_EINVAL, "create: null argument");
  if (cfg->max_slots < 1 || cfg->max_slots > 256) return fail(JXLR_EINVAL, "create: max_slots out of [1, 256]");
  if (cfg->precision != JXLR_PREC_FP32 && cfg->precision != JXLR_PREC_TC_F16X3)
    return fail(JXLR_EINVAL, "create: unsupported precision");
  int ndev = 0;
  CK(cudaGetDeviceCount(&ndev));
  if (cfg->device < 0 || cfg->device >= ndev) return fail(JXLR_EINVAL, "create: bad device");
  CK(cudaSetDevice(cfg->device));

  // constant tables (host, double precision -> float)
  std::vector<float> raw(kDequantFloats), scaled(kDequantFloats);
  if (!default_dequant(raw.data())) return fail(JXLR_EINVAL, "default dequant matrices ill-formed");
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
    return fail(JXLR_ECUDA, "create: constant upload failed");
  std::vector<float> lf_up(kLfUpFloats), lf_inv(kLfInvFloats);
  float lf_half = 0.f;
  lf_tables(lf_up.data(), lf_inv.data(), &lf_half);
  if (!upload_lf_constants(lf_up.data(), lf_inv.data(), lf_half))
    return fail(JXLR_ECUDA, "create: constant upload failed");
  {
    // odd parts of the unscaled 8- and 4-point inverse DCT (M.6.2)
    const double pi = 3.14159265358979323846;
    float odd8[16], odd4[4];
    for (int n = 0; n < 4; ++n)
      for (int j = 0; j < 4; ++j)
        odd8[n * 4 + j] = static_cast<float>(std::cos((2 * n + 1) * (2 * j + 1) * pi / 16.0));
    for (int n = 0; n < 2; ++n)
      for (int j = 0; j < 2; ++j)
        odd4[n * 2 + j] = static_cast<float>(std::cos((2 * n + 1) * (2 * j + 1) * pi / 8.0));
    if (!upload_jpeg_constants(odd8, odd4, static_cast<float>(std::cos(pi / 4.0))))
      return fail(JXLR_ECUDA, "create: constant upload failed");
  }
  {
    std::vector<uint64_t> jump(kNoiseJumpLevels * 256);
    noise_jump_tables(jump.data());
    if (!upload_noise_constants(jump.data()))
      return fail(JXLR_ECUDA, "create: constant upload failed");
  }

  auto* ctx = new jxl_recon_ctx();
  ctx->device = cfg->device;
  ctx->cap = cfg->hbm_cap_bytes;
  ctx->timing = cfg->timing != 0;
  ctx->precision = cfg->precision;
  if (const char* v = std::getenv("JXLR_RECON_VARIANT"))
    ctx->recon_variant = std::strcmp(v, "persistent") == 0 ? kReconPersistent : kReconGrid;
  cudaError_t e = cudaMalloc(&ctx->d_dequant, sizeof(float) * kDequantFloats);
  if (e == cudaSuccess)
    e = cudaMemcpy(ctx->d_dequant, scaled.data(), sizeof(float) * kDequantFloats,
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess && ctx->precision == JXLR_PREC_TC_F16X3) {
    std::vector<unsigned char> tcb(kTcBasisBytes);
    tc_basis_tables(tcb.data());
    e = cudaMalloc(&ctx->d_tcb, kTcBasisBytes);
    if (e == cudaSuccess)
      e = cudaMemcpy(ctx->d_tcb, tcb.data(), kTcBasisBytes, cudaMemcpyHostToDevice);
  }
  ctx->slots.resize(cfg->max_slots);
  // each slot: one stream per priority level of the device (at most kMaxPrio)
  int least = 0, greatest = 0;
  if (e == cudaSuccess && !cfg->cuda_stream)
    e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
  const int levels = std::min(kMaxPrio, least - greatest + 1);
  for (auto& s : ctx->slots) {
    if (cfg->cuda_stream) {
      s.stream = static_cast<cudaStream_t>(cfg->cuda_stream);
      s.own_stream = false;
    } else {
      for (int l = 0; l < levels && e == cudaSuccess; ++l)
        e = cudaStreamCreateWithPriority(&s.pstream[l], cudaStreamNonBlocking, least - l);
      if (e == cudaSuccess) {
        s.nprio = levels;
        s.stream = s.pstream[0];
      }
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
    for (auto& ev : s.ev)
      if (e == cudaSuccess) e = cudaEventCreate(&ev);
    if (e == cudaSuccess) e = cudaMallocHost(&s.h_status, kStatusWords * sizeof(unsigned));
  }
  if (e != cudaSuccess) {
    jxl_recon_destroy(ctx);
    return cuda_fail(e, "create");
  }
  *out = ctx;
  return JXLR_OK;
}

jxlr_status jxl_recon_destroy(jxl_recon_ctx* ctx) {
  if (!ctx) return JXLR_OK;
  cudaSetDevice(ctx->device);
  for (auto& s : ctx->slots) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    if (s.arena) {
      cudaFreeAsync(s.arena, s.stream);
      cudaStreamSynchronize(s.stream);
    }
    if (s.h_status) cudaFreeHost(s.h_status);
    for (auto& ev : s.ev)
      if (ev) cudaEventDestroy(ev);
    if (s.done) cudaEventDestroy(s.done);
    if (s.own_stream)
      for (int l = 0; l < s.nprio; ++l)
        if (s.pstream[l]) cudaStreamDestroy(s.pstream[l]);
  }
  if (ctx->d_dequant) cudaFree(ctx->d_dequant);
  if (ctx->d_tcb) cudaFree(ctx->d_tcb);
  delete ctx;
  return JXLR_OK;
}

}  // extern "C"

namespace {

// Host-side check of a DctSelect map (C.5.4): every block is covered by
// exactly one naturally aligned, in-bounds varblock.
bool host_map_valid(const uint8_t* vmap, int bw, int bh, std::string* why) {
  std::vector<uint8_t> cov(static_cast<size_t>(bw) * bh, 0);
  for (int by = 0; by < bh; ++by) {
    for (int bx = 0; bx < bw; ++bx) {
      const unsigned code = vmap[by * bw + bx];
      if (code == kCovered) continue;
      if (code >= kNumCodes) { *why = "invalid DctSelect code"; return false; }
      const int w8 = kShapeW[code] / 8, h8 = kShapeH[code] / 8;
      if (bx % w8 || by % h8) { *why = "varblock not naturally aligned"; return false; }
      if (bx + w8 > bw || by + h8 > bh) { *why = "varblock out of bounds"; return false; }
      for (int yy = 0; yy < h8; ++yy)
        for (int xx = 0; xx < w8; ++xx) {
          if ((xx | yy) && vmap[(by + yy) * bw + bx + xx] != kCovered) {
            *why = "varblocks overlap"; return false;
          }
          cov[(by + yy) * bw + bx + xx]++;
        }
    }
  }
  for (auto c : cov)
    if (c != 1) { *why = "blocks not covered by exactly one varblock"; return false; }
  return true;
}

// The priority level of a request of `pixels` pixels: larger images get
// higher levels (one level per factor of 4 from 256 Kpx up), so that on the
// device the blocks of large requests, which set the tail latency, are
// scheduled before those of small ones, and small ones fill the SMs that
// large ones leave free.
int size_level(uint64_t pixels, int nlevels) {
  int lvl = 0;
  for (uint64_t t = uint64_t(1) << 18; pixels >= t && lvl + 1 < nlevels; t <<= 2) ++lvl;
  return lvl;
}

// Finds a free slot and makes sure its arena holds `need` bytes within the
// HBM cap; its stream is the one of the request's size class.  Called with
// ctx->mu held.
jxlr_status acquire_slot(jxl_recon_ctx* ctx, size_t need, uint64_t pixels, Slot** out) {
  Slot* fit = nullptr;   // smallest idle arena that already holds `need`
  Slot* any = nullptr;   // else the idle slot with the largest arena
  for (auto& s : ctx->slots) {
    if (s.busy) continue;
    if (s.arena_bytes >= need && (!fit || s.arena_bytes < fit->arena_bytes)) fit = &s;
    if (!any || s.arena_bytes > any->arena_bytes) any = &s;
  }
  Slot* best = fit ? fit : any;
  if (ctx->cap && need > ctx->cap) return fail(JXLR_ENOMEM, "request exceeds the HBM cap");
  if (!best) return fail(JXLR_EBUSY, "no free slot");
  // the request's stream first: the arena below is freed and allocated in
  // its order (the slot's earlier work, on whichever stream, has completed)
  if (best->nprio) best->stream = best->pstream[size_level(pixels, best->nprio)];
  if (best->arena_bytes < need) {
    const size_t others = ctx->bytes - best->arena_bytes;
    if (ctx->cap && others + need > ctx->cap) {
      // free idle arenas before refusing
      for (auto& s : ctx->slots) {
        if (!s.busy && &s != best && s.arena) {
          cudaFreeAsync(s.arena, s.stream);
          ctx->bytes -= s.arena_bytes;
          s.arena = nullptr;
          s.arena_bytes = 0;
        }
      }
      if (ctx->bytes - best->arena_bytes + need > ctx->cap)
        return fail(JXLR_EBUSY, "not enough HBM under the cap now");
    }
    // stream-ordered: growing an idle slot's arena does not synchronise the
    // device (a plain cudaFree would wait for every request in flight)
    if (best->arena) {
      cudaFreeAsync(best->arena, best->stream);
      ctx->bytes -= best->arena_bytes;
      best->arena = nullptr;
      best->arena_bytes = 0;
    }
    const size_t sz = align_up(need, size_t(1) << 20);
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&best->arena), sz, best->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(JXLR_ENOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
    }
    best->arena_bytes = sz;
    ctx->bytes += sz;
  }
  *out = best;
  return JXLR_OK;
}

struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(char* b) : base(b) {}
  template <class T>
  T* take(size_t count) {
    off = align_up(off, 256);
    T* p = reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return p;
  }
};

void mark(Slot* s, int i) {
  if (s->timed) cudaEventRecord(s->ev[i], s->stream);
}

jxlr_status finish_submit(jxl_recon_ctx* ctx, Slot* slot, unsigned* d_status, uint64_t* ticket) {
  CK(cudaMemcpyAsync(slot->h_status, d_status, kStatusWords * sizeof(unsigned), cudaMemcpyDeviceToHost,
                     slot->stream));
  CK(cudaEventRecord(slot->done, slot->stream));
  CK(cudaGetLastError());
  slot->busy = true;
  slot->ticket = ctx->next_ticket++;
  *ticket = slot->ticket;
  return JXLR_OK;
}

}  // namespace

// K.5.2 channels of every group into r ([3][ys][xs]); fa reads them.
static int setup_noise(FilterArgs& fa, float* r, cudaStream_t s) {
  NoiseGenArgs na;
  na.r = r;
  na.rs = fa.xs;
  na.ps = static_cast<size_t>(fa.xs) * fa.ys;
  na.xs = fa.xs;
  na.ys = fa.ys;
  na.ngx = (fa.xs + 255) / 256;
  na.ngy = (fa.ys + 255) / 256;
  fa.noise_r = r;
  fa.nrs = na.rs;
  fa.nps = na.ps;
  return launch_noise_gen(na, s);
}

// J.2 into eo (the blocks the sigma pass listed; it copied the others
// there), J.3 in place on eo when asked, then J.4 / L.2 (and K.5) from eo.
// fa: the filter arguments of the request (EPF on); orig = fa.xyb.  Returns
// the number of launches.
static int launch_epf_chain(Slot* slot, const FilterArgs& fa, float* eo, const EpfSink& sink,
                            bool qco, const uint8_t* vmap, const float* acmul,
                            const float* dequant, int bh, const jxl_recon_filter_params& fp,
                            cudaStream_t s) {
  const size_t wp = static_cast<size_t>(fa.bw) * 8, hp = static_cast<size_t>(bh) * 8;
  FilterArgs e = fa;
  e.epf_out = eo;
  e.ors = wp;
  e.ops = wp * hp;
  mark(slot, 5);
  launch_epf_work(e, sink.list, sink.count, sink.count + 1, s);   // status words 4, 5
  mark(slot, 6);
  slot->epf_marked = slot->timed;
  if (qco) {
    QcoArgs q;
    std::memset(&q, 0, sizeof(q));
    q.orig = fa.xyb;
    q.ors = fa.rstride;
    q.ops = fa.pstride;
    q.f = eo;
    q.frs = wp;
    q.fps = wp * hp;
    q.vmap = vmap;
    q.acmul = acmul;
    q.dequant = dequant;
    q.xs = fa.xs; q.ys = fa.ys; q.bw = fa.bw; q.bh = bh;
    for (int c = 0; c < 3; ++c) q.m_dc[c] = fp.m_dc[c];
    q.mul = fp.qco_interval_mul;
    q.vec = (q.ors % 4 == 0 && q.ops % 4 == 0 && q.frs % 4 == 0 && q.fps % 4 == 0 &&
             (reinterpret_cast<uintptr_t>(q.orig) & 15) == 0 &&
             (reinterpret_cast<uintptr_t>(q.f) & 15) == 0) ? 1 : 0;
    launch_qco(q, s);
  }
  FilterArgs g = fa;
  g.epf = 0;
  g.sigma = nullptr;
  g.xyb = eo;
  g.rstride = wp;
  g.pstride = wp * hp;
  launch_filter(g, s);
  return qco ? 3 : 2;
}

extern "C" jxlr_status jxl_recon_submit(jxl_recon_ctx* ctx, const jxl_recon_coeffs* co,
                                        const uint8_t* vmap, const float* qf,
                                        const jxl_recon_cfl* cfl,
                                        const jxl_recon_filter_params* fp,
                                        const jxl_recon_output* out, uint64_t* ticket) {
  if (!ctx || !co || !vmap || !qf || !cfl || !cfl->k || !fp || !out || !ticket)
    return fail(JXLR_EINVAL, "submit: null argument");
  const int xs = static_cast<int>(co->xsize), ys = static_cast<int>(co->ysize);
  if (xs <= 0 || ys <= 0 || xs > 65536 || ys > 65536)
    return fail(JXLR_EINVAL, "submit: image size out of [1, 65536]");
  const int wp = (xs + 7) & ~7, hp = (ys + 7) & ~7, bw = wp / 8, bh = hp / 8;
  const int tw = (wp + 63) / 64, th = (hp + 63) / 64;
  if (co->row_stride_elems < static_cast<size_t>(wp))
    return fail(JXLR_EINVAL, "submit: coefficient row stride below the padded width");
  for (int c = 0; c < 3; ++c)
    if (!co->plane[c]) return fail(JXLR_EINVAL, "submit: null coefficient plane");
  if (out->dtype < 0 || out->dtype > 3 || !out->data) return fail(JXLR_EINVAL, "submit: bad output");
  const size_t px_bytes = out->dtype == 1 ? 6 : out->dtype == 2 ? 3 : 12;
  if (out->row_stride_bytes < px_bytes * xs) return fail(JXLR_EINVAL, "submit: output stride too small");
  if (fp->epf && !fp->sharpness) return fail(JXLR_EINVAL, "submit: EPF needs the sharpness map");
  const bool dev_in = co->on_device != 0;
  if (dev_in) {
    if (co->row_stride_elems % 8) return fail(JXLR_EINVAL, "submit: device coefficient rows must be 16-byte multiples");
    for (int c = 0; c < 3; ++c)
      if (reinterpret_cast<uintptr_t>(co->plane[c]) & 15)
        return fail(JXLR_EINVAL, "submit: device coefficient planes must be 16-byte aligned");
  } else {
    std::string why;
    if (!host_map_valid(vmap, bw, bh, &why)) return fail(JXLR_EINVAL, "submit: " + why);
  }
  std::vector<float> dq_scaled;
  if (fp->dequant) {
    if (!dequant_valid(fp->dequant))
      return fail(JXLR_EINVAL, "submit: dequant matrix entry non-positive or not finite");
    dq_scaled.resize(kDequantFloats);
    prescale_dequant(fp->dequant, dq_scaled.data());
  }
  const bool filters = fp->epf || fp->gab || fp->noise;

  // ---- scratch layout ----
  const size_t cstride = wp;
  size_t need = 0;
  auto add = [&](size_t bytes) { need = align_up(need, 256) + bytes; };
  add(sizeof(unsigned) * kStatusWords);               // status
  if (!dev_in) {
    for (int c = 0; c < 3; ++c) add(sizeof(int16_t) * cstride * hp);
    add(static_cast<size_t>(bw) * bh);                // map
    add(sizeof(float) * bw * bh);                     // quant field
    add(sizeof(float) * tw * th * 2);                 // cfl
    if (fp->epf) add(static_cast<size_t>(bw) * bh);   // sharpness
  }
  if (fp->dequant) add(sizeof(float) * kDequantFloats);
  if (filters) add(sizeof(float) * 3 * wp * hp);
  if (fp->epf) add(sizeof(int16_t) * bw * bh);
  const bool dcsteps = fp->dc_smooth || fp->lf_predict;
  const size_t nblk = static_cast<size_t>(bw) * bh;
  if (dcsteps) {
    add(nblk);                                        // owner bytes
    add(sizeof(float) * 3 * nblk);                    // DC after F.2 and G
  }
  if (fp->lf_predict) {
    add(sizeof(float) * 12 * nblk);                   // DC2x2 image
    add(sizeof(float) * 12 * nblk);                   // predicted coefficients
  }
  const bool qco = fp->epf && fp->qco;
  if (fp->epf) {
    add(sizeof(float) * 3 * wp * hp);                 // J.2 output
    add(sizeof(int) * nblk);                          // blocks J.2 filters
  }
  if (fp->noise) add(sizeof(float) * 3 * static_cast<size_t>(xs) * ys);   // K.5.2 channels
  const size_t out_bytes = out->row_stride_bytes * (ys - 1) + px_bytes * xs;
  if (!out->on_device) add(out_bytes);
  need = align_up(need, 256);

  std::lock_guard<std::mutex> lock(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  Slot* slot = nullptr;
  jxlr_status st = acquire_slot(ctx, need, static_cast<uint64_t>(xs) * static_cast<uint64_t>(ys), &slot);
  if (st != JXLR_OK) return st;
  slot->timed = ctx->timing;
  slot->epf_marked = false;
  slot->t_submit = Clock::now();
  cudaStream_t s = slot->stream;
  Carve cv(slot->arena);
  unsigned* d_status = cv.take<unsigned>(kStatusWords);
  CK(cudaMemsetAsync(d_status, 0, kStatusWords * sizeof(unsigned), s));
  mark(slot, 0);

  ReconArgs ra;
  std::memset(&ra, 0, sizeof(ra));
  const uint8_t* d_sharp = fp->sharpness;
  if (!dev_in) {
    for (int c = 0; c < 3; ++c) {
      int16_t* d = cv.take<int16_t>(cstride * hp);
      CK(cudaMemcpy2DAsync(d, cstride * 2, co->plane[c], co->row_stride_elems * 2, wp * 2, hp,
                           cudaMemcpyHostToDevice, s));
      ra.coef[c] = d;
    }
    uint8_t* dm = cv.take<uint8_t>(static_cast<size_t>(bw) * bh);
    CK(cudaMemcpyAsync(dm, vmap, static_cast<size_t>(bw) * bh, cudaMemcpyHostToDevice, s));
    float* dq = cv.take<float>(static_cast<size_t>(bw) * bh);
    CK(cudaMemcpyAsync(dq, qf, sizeof(float) * bw * bh, cudaMemcpyHostToDevice, s));
    float* dc = cv.take<float>(static_cast<size_t>(tw) * th * 2);
    CK(cudaMemcpyAsync(dc, cfl->k, sizeof(float) * tw * th * 2, cudaMemcpyHostToDevice, s));
    ra.vmap = dm;
    ra.acmul = dq;
    ra.cfl = dc;
    ra.cstride = cstride;
    if (fp->epf) {
      uint8_t* ds = cv.take<uint8_t>(static_cast<size_t>(bw) * bh);
      CK(cudaMemcpyAsync(ds, fp->sharpness, static_cast<size_t>(bw) * bh, cudaMemcpyHostToDevice, s));
      d_sharp = ds;
    }
  } else {
    for (int c = 0; c < 3; ++c) ra.coef[c] = co->plane[c];
    ra.cstride = co->row_stride_elems;
    ra.vmap = vmap;
    ra.acmul = qf;
    ra.cfl = cfl->k;
  }
  mark(slot, 1);
  if (dev_in) {
    launch_validate(ra.vmap, bw, bh, d_status, s);
    ctx->launches++;
  }
  mark(slot, 2);
  if (fp->dequant) {
    float* d = cv.take<float>(kDequantFloats);
    CK(cudaMemcpyAsync(d, dq_scaled.data(), sizeof(float) * kDequantFloats, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));   // dq_scaled is a local buffer
    ra.dequant = d;
  } else {
    ra.dequant = ctx->d_dequant;
  }
  ra.sharp = d_sharp;
  ra.xs = xs; ra.ys = ys; ra.wp = wp; ra.hp = hp; ra.bw = bw; ra.bh = bh; ra.tw = tw;
  for (int c = 0; c < 3; ++c) {
    ra.m_dc[c] = fp->m_dc[c];
    ra.one_minus_bias[c] = one_minus_bias(c);
  }
  ra.kx_dc = cfl->kx_dc;
  ra.kb_dc = cfl->kb_dc;
  ra.sp = sigma_params(*fp);
  ra.cp = color_params(*fp);
  ra.tcb = ctx->d_tcb;
  ra.err = d_status + 3;
  const bool tc = ctx->precision == JXLR_PREC_TC_F16X3;
  if (dcsteps) {
    LfArgs la;
    std::memset(&la, 0, sizeof(la));
    for (int c = 0; c < 3; ++c) {
      la.coef[c] = ra.coef[c];
      la.m_dc[c] = fp->m_dc[c];
    }
    la.cstride = ra.cstride;
    la.vmap = ra.vmap;
    la.bw = bw;
    la.bh = bh;
    la.bpl = nblk;
    la.kx_dc = cfl->kx_dc;
    la.kb_dc = cfl->kb_dc;
    la.smooth = fp->dc_smooth != 0;
    la.predict = fp->lf_predict != 0;
    la.own = cv.take<uint8_t>(nblk);
    la.d1 = cv.take<float>(3 * nblk);
    if (la.predict) {
      la.u = cv.take<float>(12 * nblk);
      la.us = cv.take<float>(12 * nblk);
    }
    ctx->launches += launch_lf(la, s);
    ra.dc1 = la.d1;
    ra.lfp = la.us;
  }

  OutParams op;
  char* d_out = nullptr;
  if (out->on_device) {
    op.data = out->data;
  } else {
    d_out = cv.take<char>(out_bytes);
    op.data = d_out;
  }
  op.stride = out->row_stride_bytes;
  op.dtype = out->dtype;

  if (filters) {
    float* xyb = cv.take<float>(static_cast<size_t>(3) * wp * hp);
    int16_t* sig = fp->epf ? cv.take<int16_t>(static_cast<size_t>(bw) * bh) : nullptr;
    EpfSink sink;
    std::memset(&sink, 0, sizeof(sink));
    float* eo = nullptr;
    if (fp->epf) {
      eo = cv.take<float>(static_cast<size_t>(3) * wp * hp);
      sink.list = cv.take<int>(nblk);
      sink.count = d_status + 4;
      sink.pass = eo;
      sink.prs = wp;
      sink.pps = static_cast<size_t>(wp) * hp;
    }
    ra.write_xyb = 1;
    ra.xyb = xyb;
    ra.sigma = sig;
    ra.epf = sink;
    if (tc) launch_recon_tc(ra, s);
    else launch_recon(ra, s, ctx->recon_variant);
    ctx->launches++;
    mark(slot, 3);
    FilterArgs fa = filter_args(*fp);
    fa.err = d_status + 3;
    fa.xyb = xyb;
    fa.rstride = wp;
    fa.pstride = static_cast<size_t>(wp) * hp;
    fa.xs = xs; fa.ys = ys; fa.bw = bw;
    fa.sigma = sig;
    fa.out = op;
    if (fp->noise) ctx->launches += setup_noise(fa, cv.take<float>(3 * static_cast<size_t>(xs) * ys), s);
    if (fp->epf) {
      ctx->launches += launch_epf_chain(slot, fa, eo, sink, qco, ra.vmap, ra.acmul, ra.dequant,
                                        bh, *fp, s);
    } else {
      launch_filter(fa, s);
      ctx->launches++;
    }
  } else {
    ra.write_xyb = 0;
    ra.out = op;
    if (tc) launch_recon_tc(ra, s);
    else launch_recon(ra, s, ctx->recon_variant);
    ctx->launches++;
    mark(slot, 3);
  }
  mark(slot, 4);
  if (!out->on_device)
    CK(cudaMemcpy2DAsync(out->data, out->row_stride_bytes, d_out, out->row_stride_bytes,
                         px_bytes * xs, ys, cudaMemcpyDeviceToHost, s));
  slot->check_status = dev_in;
  return finish_submit(ctx, slot, d_status, ticket);
}

extern "C" jxlr_status jxl_recon_submit_xyb(jxl_recon_ctx* ctx, const float* xyb, uint32_t xsize,
                                            uint32_t ysize, size_t row_stride_elems,
                                            const uint8_t* vmap, const float* qf,
                                            const jxl_recon_filter_params* fp,
                                            const jxl_recon_output* out, uint64_t* ticket) {
  if (!ctx || !xyb || !fp || !out || !ticket) return fail(JXLR_EINVAL, "submit_xyb: null argument");
  const int xs = static_cast<int>(xsize), ys = static_cast<int>(ysize);
  if (xs <= 0 || ys <= 0 || xs > 65536 || ys > 65536)
    return fail(JXLR_EINVAL, "submit_xyb: image size out of [1, 65536]");
  if (row_stride_elems < static_cast<size_t>(xs)) return fail(JXLR_EINVAL, "submit_xyb: row stride");
  if (fp->epf && (!vmap || !qf || !fp->sharpness))
    return fail(JXLR_EINVAL, "submit_xyb: EPF needs the map, quant field and sharpness");
  if (out->dtype < 0 || out->dtype > 3 || !out->data || !out->on_device)
    return fail(JXLR_EINVAL, "submit_xyb: output must be a device buffer");
  const int bw = (xs + 7) / 8, bh = (ys + 7) / 8;
  const bool qco = fp->epf && fp->qco;
  if (qco && fp->dequant)
    return fail(JXLR_EINVAL, "submit_xyb: the quantization constraint uses the default matrices here");
  size_t need = 256 + (fp->epf ? align_up(sizeof(int16_t) * bw * bh, 256) : 0);
  if (fp->epf) {
    need += align_up(sizeof(float) * 3 * 64 * static_cast<size_t>(bw) * bh, 256);
    need += align_up(sizeof(int) * static_cast<size_t>(bw) * bh, 256);
  }
  if (fp->noise) need += align_up(sizeof(float) * 3 * static_cast<size_t>(xs) * ys, 256);
  std::lock_guard<std::mutex> lock(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  Slot* slot = nullptr;
  jxlr_status st = acquire_slot(ctx, need, static_cast<uint64_t>(xs) * static_cast<uint64_t>(ys), &slot);
  if (st != JXLR_OK) return st;
  slot->timed = ctx->timing;
  slot->epf_marked = false;
  slot->t_submit = Clock::now();
  cudaStream_t s = slot->stream;
  Carve cv(slot->arena);
  unsigned* d_status = cv.take<unsigned>(kStatusWords);
  CK(cudaMemsetAsync(d_status, 0, kStatusWords * sizeof(unsigned), s));
  mark(slot, 0);
  mark(slot, 1);   // no input staging on this path
  int16_t* sig = nullptr;
  EpfSink sink;
  std::memset(&sink, 0, sizeof(sink));
  float* eo = nullptr;
  if (fp->epf) {
    launch_validate(vmap, bw, bh, d_status, s);
    ctx->launches++;
  }
  mark(slot, 2);
  if (fp->epf) {
    sig = cv.take<int16_t>(static_cast<size_t>(bw) * bh);
    eo = cv.take<float>(static_cast<size_t>(3) * 64 * bw * bh);
    sink.list = cv.take<int>(static_cast<size_t>(bw) * bh);
    sink.count = d_status + 4;
    sink.pass = eo;
    sink.prs = static_cast<size_t>(8) * bw;
    sink.pps = static_cast<size_t>(64) * bw * bh;
    SigmaArgs sa;
    std::memset(&sa, 0, sizeof(sa));
    sa.xyb = xyb;
    sa.rstride = row_stride_elems;
    sa.pstride = row_stride_elems * ys;
    sa.vmap = vmap;
    sa.acmul = qf;
    sa.sharp = fp->sharpness;
    sa.xs = xs; sa.ys = ys; sa.bw = bw; sa.bh = bh;
    sa.sigma = sig;
    sa.sp = sigma_params(*fp);
    sa.epf = sink;
    launch_sigma(sa, s);
    ctx->launches++;
  }
  mark(slot, 3);
  FilterArgs fa = filter_args(*fp);
  fa.err = d_status + 3;
  fa.xyb = xyb;
  fa.rstride = row_stride_elems;
  fa.pstride = row_stride_elems * ys;
  fa.xs = xs; fa.ys = ys; fa.bw = bw;
  fa.sigma = sig;
  fa.out.data = out->data;
  fa.out.stride = out->row_stride_bytes;
  fa.out.dtype = out->dtype;
  if (fp->noise) ctx->launches += setup_noise(fa, cv.take<float>(3 * static_cast<size_t>(xs) * ys), s);
  if (fp->epf) {
    ctx->launches += launch_epf_chain(slot, fa, eo, sink, qco, vmap, qf, ctx->d_dequant, bh, *fp,
                                      s);
  } else {
    launch_filter(fa, s);
    ctx->launches++;
  }
  mark(slot, 4);
  slot->check_status = fp->epf != 0;
  return finish_submit(ctx, slot, d_status, ticket);
}

extern "C" jxlr_status jxl_recon_poll(jxl_recon_ctx* ctx, uint64_t ticket, int64_t timeout_us,
                                      double* latency_ms) {
  if (!ctx) return fail(JXLR_EINVAL, "poll: null context");
  Slot* slot = nullptr;
  {
    std::lock_guard<std::mutex> lock(ctx->mu);
    for (auto& s : ctx->slots)
      if (s.busy && s.ticket == ticket) slot = &s;
  }
  if (!slot) return fail(JXLR_EINVAL, "poll: unknown or already completed ticket");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(JXLR_ECUDA, "poll: set device");
  const auto t0 = Clock::now();
  cudaError_t q;
  if (timeout_us < 0) {
    q = cudaEventSynchronize(slot->done);
  } else {
    for (;;) {
      q = cudaEventQuery(slot->done);
      if (q != cudaErrorNotReady) break;
      const auto us = std::chrono::duration_cast<std::chrono::microseconds>(Clock::now() - t0).count();
      if (us >= timeout_us) return timeout_us == 0 ? JXLR_EAGAIN : JXLR_ETIMEDOUT;
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  }
  const auto t1 = Clock::now();
  std::lock_guard<std::mutex> lock(ctx->mu);
  slot->busy = false;
  if (q != cudaSuccess) return cuda_fail(q, "poll");
  if (latency_ms)
    *latency_ms = std::chrono::duration<double, std::milli>(t1 - slot->t_submit).count();
  if (slot->timed) {
    Timing t;
    float a = 0, b = 0, c = 0, d = 0;
    cudaEventElapsedTime(&a, slot->ev[0], slot->ev[1]);
    cudaEventElapsedTime(&b, slot->ev[1], slot->ev[2]);
    cudaEventElapsedTime(&c, slot->ev[2], slot->ev[3]);
    cudaEventElapsedTime(&d, slot->ev[3], slot->ev[4]);
    t.ms[0] = b;   // validation
    t.ms[1] = c;   // dequantisation + transforms (+ colour when unfiltered)
    t.ms[2] = d;   // filters + colour
    t.ms[3] = a;   // input staging copies
    if (slot->epf_marked) {
      cudaEventElapsedTime(&t.epf_ms, slot->ev[5], slot->ev[6]);
      t.epf_blocks = slot->h_status[4];
    }
    if (ctx->timings.size() > 4096) ctx->timings.clear();
    ctx->timings[ticket] = t;
  }
  if (slot->h_status[3] != 0)
    return fail(JXLR_ETIMEDOUT, (slot->h_status[3] & 8u)
                                    ? "tile-load wait expired in the filter kernel"
                                    : "tensor-core completion wait expired in the transform kernel");
  if (slot->check_status && slot->h_status[0] != 0) {
    char buf[96];
    std::snprintf(buf, sizeof(buf), "device validation: DctSelect map ill-formed (flags 0x%x)",
                  slot->h_status[0]);
    return fail(JXLR_EINVAL, buf);
  }
  return JXLR_OK;
}

extern "C" jxlr_status jxl_recon_stage_ms(jxl_recon_ctx* ctx, uint64_t ticket, float ms[4]) {
  if (!ctx || !ms) return fail(JXLR_EINVAL, "stage_ms: null argument");
  std::lock_guard<std::mutex> lock(ctx->mu);
  auto it = ctx->timings.find(ticket);
  if (it == ctx->timings.end()) return fail(JXLR_EINVAL, "stage_ms: no timing for this ticket");
  std::memcpy(ms, it->second.ms, sizeof(float) * 4);
  return JXLR_OK;
}

extern "C" jxlr_status jxl_recon_epf_stats(jxl_recon_ctx* ctx, uint64_t ticket, float* epf_ms,
                                           uint32_t* epf_blocks) {
  if (!ctx || !epf_ms || !epf_blocks) return fail(JXLR_EINVAL, "epf_stats: null argument");
  std::lock_guard<std::mutex> lock(ctx->mu);
  auto it = ctx->timings.find(ticket);
  if (it == ctx->timings.end()) return fail(JXLR_EINVAL, "epf_stats: no timing for this ticket");
  *epf_ms = it->second.epf_ms;
  *epf_blocks = it->second.epf_blocks;
  return JXLR_OK;
}

// ---------------------------------------------------------------------------
// JPEG1 direct rasterisation (M.6)
// ---------------------------------------------------------------------------
extern "C" jxlr_status jxl_recon_submit_jpeg(jxl_recon_ctx* ctx, const jxl_jpeg_stream* st,
                                             const jxl_recon_output* out, uint64_t* ticket) {
  if (!ctx || !st || !out || !ticket) return fail(JXLR_EINVAL, "submit_jpeg: null argument");
  const int xs = static_cast<int>(st->xsize), ys = static_cast<int>(st->ysize);
  if (xs <= 0 || ys <= 0 || xs > 65536 || ys > 65536)
    return fail(JXLR_EINVAL, "submit_jpeg: image size out of [1, 65536]");
  const int nc = static_cast<int>(st->num_components);
  if (nc != 1 && nc != 3) return fail(JXLR_EINVAL, "submit_jpeg: 1 or 3 components");
  if (out->dtype < 0 || out->dtype > 2 || !out->data)
    return fail(JXLR_EINVAL, "submit_jpeg: output must be f32, f16 or u8");
  const size_t px_bytes = out->dtype == 1 ? 6 : out->dtype == 2 ? 3 : 12;
  if (out->row_stride_bytes < px_bytes * xs) return fail(JXLR_EINVAL, "submit_jpeg: output stride too small");
  int hmax = 1, vmax = 1;
  for (int c = 0; c < nc; ++c) {
    const jxl_jpeg_component& k = st->comp[c];
    if (k.h_samp < 1 || k.h_samp > 2 || k.v_samp < 1 || k.v_samp > 2)
      return fail(JXLR_EINVAL, "submit_jpeg: sampling factors must be 1 or 2");
    hmax = std::max(hmax, static_cast<int>(k.h_samp));
    vmax = std::max(vmax, static_cast<int>(k.v_samp));
  }
  for (int c = 0; c < nc; ++c) {
    const jxl_jpeg_component& k = st->comp[c];
    if (!k.coeffs || !k.quant) return fail(JXLR_EINVAL, "submit_jpeg: null coefficients or table");
    if (k.width_in_blocks == 0 || k.height_in_blocks == 0 || k.width_in_blocks > 8192 ||
        k.height_in_blocks > 8192)
      return fail(JXLR_EINVAL, "submit_jpeg: block grid out of [1, 8192]");
    const long long cw = 8LL * k.width_in_blocks * (hmax / k.h_samp);
    const long long ch = 8LL * k.height_in_blocks * (vmax / k.v_samp);
    if (cw < xs || ch < ys) return fail(JXLR_EINVAL, "submit_jpeg: block grid does not cover the image");
    if (st->on_device && (reinterpret_cast<uintptr_t>(k.coeffs) & 15))
      return fail(JXLR_EINVAL, "submit_jpeg: device coefficients must be 16-byte aligned");
    if (k.cond && (k.quant[0] == 0 || !std::isfinite(k.cond_max_gap) || !std::isfinite(k.cond_min_step)))
      return fail(JXLR_EINVAL, "submit_jpeg: bad conditioning parameters");
    if (k.gab && !(k.gab_limit >= 0 && std::isfinite(k.gab_w1) && std::isfinite(k.gab_w2) &&
                   std::isfinite(k.gab_threshold) && 1.0 + 4.0 * k.gab_w1 + 4.0 * k.gab_w2 != 0.0))
      return fail(JXLR_EINVAL, "submit_jpeg: bad Gaborish side channel");
  }

  size_t need = 0;
  auto add = [&](size_t bytes) { need = align_up(need, 256) + bytes; };
  add(sizeof(unsigned) * kStatusWords);
  for (int c = 0; c < nc; ++c) {
    const size_t nb = static_cast<size_t>(st->comp[c].width_in_blocks) * st->comp[c].height_in_blocks;
    if (!st->on_device) add(nb * 128);
    add(nb * 256);                                    // sample plane
    if (st->comp[c].gab) add(nb * 256);               // after M.6.3
    if (st->comp[c].cond) {                           // M.6.1.1 results
      for (int k = 0; k < 4; ++k) add(nb * 4);
      add(nb);
      add(nb);
    }
  }
  const size_t out_bytes = out->row_stride_bytes * (ys - 1) + px_bytes * xs;
  if (!out->on_device) add(out_bytes);
  need = align_up(need, 256);

  std::lock_guard<std::mutex> lock(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  Slot* slot = nullptr;
  jxlr_status status = acquire_slot(ctx, need, static_cast<uint64_t>(xs) * static_cast<uint64_t>(ys), &slot);
  if (status != JXLR_OK) return status;
  slot->timed = ctx->timing;
  slot->epf_marked = false;
  slot->t_submit = Clock::now();
  cudaStream_t s = slot->stream;
  Carve cv(slot->arena);
  unsigned* d_status = cv.take<unsigned>(kStatusWords);
  CK(cudaMemsetAsync(d_status, 0, kStatusWords * sizeof(unsigned), s));
  mark(slot, 0);
  const int16_t* coef[3] = {nullptr, nullptr, nullptr};
  for (int c = 0; c < nc; ++c) {
    const size_t nb = static_cast<size_t>(st->comp[c].width_in_blocks) * st->comp[c].height_in_blocks;
    if (st->on_device) {
      coef[c] = st->comp[c].coeffs;
    } else {
      int16_t* d = cv.take<int16_t>(nb * 64);
      CK(cudaMemcpyAsync(d, st->comp[c].coeffs, nb * 128, cudaMemcpyHostToDevice, s));
      coef[c] = d;
    }
  }
  mark(slot, 1);
  mark(slot, 2);
  JpegColorArgs ca;
  std::memset(&ca, 0, sizeof(ca));
  for (int c = 0; c < nc; ++c) {
    const jxl_jpeg_component& k = st->comp[c];
    const int bw = static_cast<int>(k.width_in_blocks), bh = static_cast<int>(k.height_in_blocks);
    JpegIdctArgs ia;
    ia.coef = coef[c];
    ia.bw = bw;
    ia.bh = bh;
    // M.6.1 I(8,u) I(8,v) times the scale of the unscaled cosine sums:
    // I(8,u) S_8(u) = eps(u) / 2 with eps(0) = sqrt(1/2)
    for (int u = 0; u < 8; ++u)
      for (int v = 0; v < 8; ++v) {
        const double eu = u == 0 ? std::sqrt(0.5) : 1.0, ev = v == 0 ? std::sqrt(0.5) : 1.0;
        ia.dq[8 * u + v] = static_cast<float>(k.quant[8 * u + v] * eu * ev / 4.0);
      }
    ia.plane = cv.take<float>(static_cast<size_t>(bw) * bh * 64);
    ia.cond = 0;
    std::memset(&ia.c, 0, sizeof(ia.c));
    if (k.cond) {
      const size_t nb = static_cast<size_t>(bw) * bh;
      JpegCondArgs ja;
      ja.coef = coef[c];
      ja.bw = bw;
      ja.bh = bh;
      ja.q_h = static_cast<float>(k.quant[1]) / static_cast<float>(k.quant[0]);
      ja.q_v = static_cast<float>(k.quant[8]) / static_cast<float>(k.quant[0]);
      ja.max_gap = k.cond_max_gap;
      ja.min_step = k.cond_min_step;
      ja.out.h_approx = cv.take<float>(nb);
      ja.out.h_slope = cv.take<float>(nb);
      ja.out.v_approx = cv.take<float>(nb);
      ja.out.v_slope = cv.take<float>(nb);
      ja.out.has_h = cv.take<uint8_t>(nb);
      ja.out.has_v = cv.take<uint8_t>(nb);
      ctx->launches += launch_jpeg_cond(ja, s);
      ia.cond = 1;
      ia.c = ja.out;
      ia.m0 = static_cast<float>(k.quant[0] / 8.0);
      ia.m1 = static_cast<float>(k.quant[0] / 8.0 / std::cos(3.14159265358979323846 / 16.0));
    }
    launch_jpeg_idct(ia, s);
    ctx->launches++;
    const float* plane = ia.plane;
    if (k.gab) {
      JpegGabArgs ga;
      ga.src = ia.plane;
      ga.dst = cv.take<float>(static_cast<size_t>(bw) * bh * 64);
      ga.bw = bw;
      ga.bh = bh;
      const double norm = 1.0 + 4.0 * k.gab_w1 + 4.0 * k.gab_w2;
      ga.w0n = static_cast<float>(1.0 / norm);
      ga.w1n = static_cast<float>(k.gab_w1 / norm);
      ga.w2n = static_cast<float>(k.gab_w2 / norm);
      ga.threshold = k.gab_threshold;
      ga.limit = k.gab_limit;
      launch_jpeg_gab(ga, s);
      ctx->launches++;
      plane = ga.dst;
    }
    ca.p[c].data = plane;
    ca.p[c].w = 8 * bw;
    ca.p[c].h = 8 * bh;
    ca.p[c].up_x = static_cast<int>(k.h_samp) != hmax;
    ca.p[c].up_y = static_cast<int>(k.v_samp) != vmax;
  }
  mark(slot, 3);
  ca.ncomp = nc;
  ca.xs = xs;
  ca.ys = ys;
  char* d_out = nullptr;
  if (out->on_device) {
    ca.out = out->data;
  } else {
    d_out = cv.take<char>(out_bytes);
    ca.out = d_out;
  }
  ca.stride = out->row_stride_bytes;
  ca.dtype = out->dtype;
  launch_jpeg_color(ca, s);
  ctx->launches++;
  mark(slot, 4);
  if (!out->on_device)
    CK(cudaMemcpy2DAsync(out->data, out->row_stride_bytes, d_out, out->row_stride_bytes,
                         px_bytes * xs, ys, cudaMemcpyDeviceToHost, s));
  slot->check_status = false;
  return finish_submit(ctx, slot, d_status, ticket);
}
