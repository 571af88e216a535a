// C ABI of libcusten_gb: plan life cycle (Create / Compute / Swap / Destroy, Sec. 3),
// validation, error reporting, CUDA-graph replay and the autotuner driver.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "cs_internal.h"

namespace cs {

namespace {
thread_local std::string t_last_error;
std::atomic<int64_t> g_launches{0};
}  // namespace

int set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_last_error = buf;
  return code;
}

int cuda_error(cudaError_t e, const char* what) {
  return set_error(CS_ECUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (cached[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    cached[dev] = n;
  }
  return cached[dev];
}

}  // namespace cs

namespace cs {
namespace autotune_detail {
// Reads a 256 MB buffer (twice the L2) so the next launch starts with a cold cache; used by
// the autotuner so that candidates are timed the way they run on data larger than the L2.
__global__ void k_read_flush(const float4* __restrict__ buf, size_t n, float* __restrict__ sink) {
  float acc = 0.f;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const float4 v = buf[i];
    acc += v.x + v.y + v.z + v.w;
  }
  if (acc == 12345.678f) *sink = acc;  // keeps the loads; never true for a zeroed buffer
}

struct FlushBuffer {
  float4* buf = nullptr;
  float* sink = nullptr;
  size_t n = 0;
  int dev = -1;
};

int flush_l2(cudaStream_t s) {
  static FlushBuffer fb;  // one per process (first device that autotunes); freed at exit
  int dev = 0;
  CS_CUDA_TRY(cudaGetDevice(&dev));
  if (fb.dev != dev) {
    if (fb.buf) return CS_OK;  // autotuning on a second device times without the flush
    const size_t bytes = size_t(256) << 20;
    CS_CUDA_TRY(cudaMalloc(&fb.buf, bytes));
    CS_CUDA_TRY(cudaMalloc(&fb.sink, sizeof(float)));
    CS_CUDA_TRY(cudaMemset(fb.buf, 0, bytes));
    fb.n = bytes / sizeof(float4);
    fb.dev = dev;
  }
  k_read_flush<<<num_sms() * 4, 256, 0, s>>>(fb.buf, fb.n, fb.sink);
  CS_CUDA_TRY(cudaGetLastError());
  return CS_OK;
}

}  // namespace autotune_detail
}  // namespace cs

enum PlanKind { kStencil2D = 1, kBatch1D = 2, kCahnHilliard = 3, kStencil2DHost = 4, kWeno = 5, kCHBand = 6 };

// Band slots of a host-resident (out-of-core) 2D plan: one being copied in, one swept, one
// copied out.
constexpr int kRingSlots = 3;

struct cs_plan {
  int kind;
  const void* d_in;
  void* d_out;
  size_t elem_bytes;
  int64_t elems;  // elements in one field / packed buffer
  cs::Stencil2DConfig s2;
  cs::Batch1DConfig b1;
  cs::CHPlan* ch;
  cs::CHBand* chb;
  // graph replay
  int use_graph;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  int graph_kernels;
  // banded host-buffer path: copy-in and copy-out streams, events (created on first use)
  cudaStream_t band_stream[2];
  cudaEvent_t band_event[2 * 32 + 2];
  int band_ready;
  // host-resident 2D plan: the grid lives in host memory and streams through kRingSlots device
  // band slots of ring_ny rows each (kRingTop halo rows, ring_rows band rows, kRingBottom rows)
  int64_t ring_rows, ring_ny;
  void* ring_in[kRingSlots];
  void* ring_out[kRingSlots];
  cs::Stencil2DConfig* ring_cfg;  // kRingSlots copies of s2 with ny = ring_ny (own tensor maps)
  int64_t ring_bytes;
  // WENO advection plan: d_in = C, d_out = the advection term, plus the two velocity fields
  cs::WenoConfig weno;
  const void* d_u;
  const void* d_v;
};

namespace {

using namespace cs;

bool overlaps(const void* a, const void* b, size_t bytes) {
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  return pa < pb + bytes && pb < pa + bytes;
}

void drop_graph(cs_plan* p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->exec = nullptr;
  p->graph = nullptr;
}

int launch_direct(cs_plan* p, cudaStream_t s) {
  switch (p->kind) {
    case kStencil2D: return stencil2d_launch(&p->s2, p->d_in, p->d_out, s);
    case kBatch1D: return batch1d_launch(&p->b1, p->d_in, p->d_out, s);
    case kWeno: return weno_launch(&p->weno, p->d_in, p->d_u, p->d_v, p->d_out, s);
    case kStencil2DHost: return set_error(CS_EINVAL, "a host-resident plan computes through cs_compute_host");
    default: return set_error(CS_EINVAL, "cs_compute: not a stencil plan");
  }
}

int validate_desc_common(const cs_stencil_desc* d) {
  if (!d) return set_error(CS_EINVAL, "null stencil description");
  if (d->dtype != CS_F64 && d->dtype != CS_F32) return set_error(CS_EINVAL, "dtype must be CS_F64 or CS_F32");
  if (d->bc != CS_BC_PERIODIC && d->bc != CS_BC_NONPERIODIC) return set_error(CS_EINVAL, "bc must be periodic or non-periodic");
  if (d->dir != CS_DIR_X && d->dir != CS_DIR_Y && d->dir != CS_DIR_XY) return set_error(CS_EINVAL, "dir must be X, Y or XY");
  if (d->left < 0 || d->right < 0 || d->top < 0 || d->bottom < 0 || d->left > CS_MAX_EXTENT ||
      d->right > CS_MAX_EXTENT || d->top > CS_MAX_EXTENT || d->bottom > CS_MAX_EXTENT)
    return set_error(CS_EINVAL, "stencil extents must be in [0, %d]", CS_MAX_EXTENT);
  if (d->dir == CS_DIR_X && (d->top != 0 || d->bottom != 0))
    return set_error(CS_EINVAL, "an X stencil has top = bottom = 0");
  if (d->dir == CS_DIR_Y && (d->left != 0 || d->right != 0))
    return set_error(CS_EINVAL, "a Y stencil has left = right = 0");
  if (d->fn == CS_FN_NONE) {
    if (!d->weights) return set_error(CS_EINVAL, "weights are required when fn = CS_FN_NONE");
  } else {
    int L, R, T, B, dir;
    switch (d->fn) {
      case CS_FN_CENTRAL_D2X: L = R = 1; T = B = 0; dir = CS_DIR_X; break;
      case CS_FN_CH_NONLIN_LAP:
      case CS_FN_CUBIC_MINUS_LAP: L = R = T = B = 1; dir = CS_DIR_XY; break;
      default: return set_error(CS_EINVAL, "unknown user function %d", d->fn);
    }
    if (d->weights) return set_error(CS_EINVAL, "weights must be NULL for a user function");
    if (d->left != L || d->right != R || d->top != T || d->bottom != B || d->dir != dir)
      return set_error(CS_EINVAL, "extents / direction must match the function's footprint (%d,%d,%d,%d)", L, R, T, B);
    if (!d->coe || d->num_coe < 1 || d->num_coe > 8)
      return set_error(CS_EINVAL, "user function needs 1..8 coefficients");
  }
  return CS_OK;
}

// Host-buffer compute of a 2D plan in row bands, so that the copy in of later bands, the sweep
// of a band and the copy out of earlier bands overlap (the host link carries both directions at
// once).  A band's sweep waits for the bands its halo reaches into; with periodic rows the last
// band is copied first, since the first band's halo wraps into it.
constexpr size_t kBandMinBytes = size_t(16) << 20;
constexpr int kMaxBands = 32;

int compute_host_banded(cs_plan* p, const void* h_in, void* h_out, cudaStream_t s) {
  const Stencil2DConfig& c = p->s2;
  if (!p->band_ready) {
    for (int i = 0; i < 2; ++i) CS_CUDA_TRY(cudaStreamCreateWithFlags(&p->band_stream[i], cudaStreamNonBlocking));
    for (auto& e : p->band_event) CS_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    p->band_ready = 1;
  }
  const int64_t ny = c.ny, row_bytes = c.nx * static_cast<int64_t>(p->elem_bytes);
  // bands of about 8 MB (enough to amortise a copy call), between 2 and kMaxBands of them
  const int64_t want = std::max<int64_t>(2, std::min<int64_t>(kMaxBands, ny * row_bytes / (int64_t(8) << 20)));
  int64_t rows = (ny + want - 1) / want;
  rows = (rows + kStencilBandAlign - 1) / kStencilBandAlign * kStencilBandAlign;
  const int nb = static_cast<int>((ny + rows - 1) / rows);
  if (nb > kMaxBands) return set_error(CS_EINVAL, "internal: %d bands", nb);
  const bool periodic = c.bc == CS_BC_PERIODIC;
  const bool halo = c.top > 0 || c.bottom > 0;  // rows <= 64 >= any extent: neighbours only
  cudaStream_t sin = p->band_stream[0], sout = p->band_stream[1];
  cudaEvent_t* ev_in = p->band_event;             // [nb]: band copied in
  cudaEvent_t* ev_done = p->band_event + kMaxBands;  // [nb]: band computed
  cudaEvent_t ev_start = p->band_event[2 * kMaxBands], ev_end = p->band_event[2 * kMaxBands + 1];
  const char* hi = static_cast<const char*>(h_in);
  char* ho = static_cast<char*>(h_out);
  const char* di = static_cast<const char*>(p->d_in);
  char* dout = static_cast<char*>(p->d_out);
  auto band_rows = [&](int b) { return std::min<int64_t>(rows, ny - b * rows); };
  // copy-in order: the last band first when rows wrap; pos[b] = its place in that order
  int order[kMaxBands], pos[kMaxBands];
  for (int k = 0; k < nb; ++k) order[k] = periodic && halo ? (k == 0 ? nb - 1 : k - 1) : k;
  for (int k = 0; k < nb; ++k) pos[order[k]] = k;
  CS_CUDA_TRY(cudaEventRecord(ev_start, s));  // earlier work on the caller's stream first
  CS_CUDA_TRY(cudaStreamWaitEvent(sin, ev_start, 0));
  CS_CUDA_TRY(cudaStreamWaitEvent(sout, ev_start, 0));
  for (int k = 0; k < nb; ++k) {
    const int b = order[k];
    const size_t off = static_cast<size_t>(b * rows * row_bytes);
    CS_CUDA_TRY(cudaMemcpyAsync(const_cast<char*>(di) + off, hi + off, static_cast<size_t>(band_rows(b) * row_bytes),
                                cudaMemcpyHostToDevice, sin));
    CS_CUDA_TRY(cudaEventRecord(ev_in[b], sin));
  }
  for (int b = 0; b < nb; ++b) {
    int need = pos[b];  // the band itself and, with a halo, its neighbours (wrapping if periodic)
    if (halo) {
      const int lo = b > 0 ? b - 1 : (periodic ? nb - 1 : 0);
      const int up = b + 1 < nb ? b + 1 : (periodic ? 0 : nb - 1);
      need = std::max(need, std::max(pos[lo], pos[up]));
    }
    CS_CUDA_TRY(cudaStreamWaitEvent(s, ev_in[order[need]], 0));
    int rc = stencil2d_launch_rows(&p->s2, p->d_in, p->d_out, b * rows, b * rows + band_rows(b), s);
    if (rc != CS_OK) return rc;
    CS_CUDA_TRY(cudaEventRecord(ev_done[b], s));
    CS_CUDA_TRY(cudaStreamWaitEvent(sout, ev_done[b], 0));
    const size_t off = static_cast<size_t>(b * rows * row_bytes);
    CS_CUDA_TRY(cudaMemcpyAsync(ho + off, dout + off, static_cast<size_t>(band_rows(b) * row_bytes),
                                cudaMemcpyDeviceToHost, sout));
  }
  CS_CUDA_TRY(cudaEventRecord(ev_end, sout));
  CS_CUDA_TRY(cudaStreamWaitEvent(s, ev_end, 0));
  CS_CUDA_TRY(cudaStreamSynchronize(s));
  return CS_OK;
}

// Fills a 2D plan's stencil configuration from a validated description and prepares it.
int fill_2d_config(cs_plan* p, const cs_stencil_desc* d) {
  Stencil2DConfig& c = p->s2;
  c.nx = d->nx; c.ny = d->ny; c.dir = d->dir; c.bc = d->bc; c.dtype = d->dtype;
  c.left = d->left; c.right = d->right; c.top = d->top; c.bottom = d->bottom;
  c.fn = d->fn;
  c.tile_rows = 64;
  const int nw = (d->left + d->right + 1) * (d->top + d->bottom + 1);
  if (d->fn == CS_FN_NONE) {
    memcpy(c.weights, d->weights, sizeof(double) * nw);
  } else {
    c.num_coe = d->num_coe;
    memcpy(c.coe, d->coe, sizeof(double) * d->num_coe);
  }
  return stencil2d_prepare(&c);
}

// ---- host-resident (out-of-core) 2D plans --------------------------------------------------------
// The grid stays in host memory and passes through a ring of kRingSlots band slots in device
// memory (Sec. 2's y-tiles, streamed: copy in, sweep, copy out on three streams).  Slot layout:
// row kRingTop of a slot is the band's first row (a multiple of 64 in the grid, so the band's
// tiles are the grid's tiles); the rows above and below hold the halo the band's tiles read --
// the neighbouring grid rows, wrapped at the grid's ends for periodic plans and zero for
// non-periodic ones, exactly what the device sweep's tile loader stages there.  Every tile of a
// band therefore stages the same values as in a sweep of the whole grid, and the streamed result
// equals the device sweep bit for bit.
constexpr int64_t kRingTop = kStencilBandAlign;
constexpr int64_t kRingBottom = kStencilBandAlign + CS_MAX_EXTENT;  // ragged last tile + halo
constexpr int64_t kRingMinRows = 2 * kStencilBandAlign;

void ring_free(cs_plan* p) {
  for (int k = 0; k < kRingSlots; ++k) {
    cudaFree(p->ring_in[k]);
    cudaFree(p->ring_out[k]);
    p->ring_in[k] = p->ring_out[k] = nullptr;
  }
  delete[] p->ring_cfg;
  p->ring_cfg = nullptr;
}

int ring_streams(cs_plan* p) {
  if (p->band_ready) return CS_OK;
  for (int i = 0; i < 2; ++i) CS_CUDA_TRY(cudaStreamCreateWithFlags(&p->band_stream[i], cudaStreamNonBlocking));
  for (auto& e : p->band_event) CS_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  p->band_ready = 1;
  return CS_OK;
}

// Copies grid rows [g_lo, g_hi) (any integers; ny >= kRingMinRows > the widest reach, so one wrap
// at most) into slot rows starting at `slot_row`: rows inside the grid from h_in, rows outside
// wrapped (periodic) or zeroed (non-periodic).
int ring_fill(const cs_plan* p, const char* h_in, char* slot, int64_t g_lo, int64_t g_hi, int64_t slot_row,
              cudaStream_t st) {
  const int64_t ny = p->s2.ny, rb = p->s2.nx * static_cast<int64_t>(p->elem_bytes);
  const bool periodic = p->s2.bc == CS_BC_PERIODIC;
  const int64_t cuts[4] = {g_lo, std::max<int64_t>(g_lo, std::min<int64_t>(0, g_hi)),
                           std::max<int64_t>(g_lo, std::min<int64_t>(ny, g_hi)), g_hi};
  for (int part = 0; part < 3; ++part) {
    const int64_t a = std::max(cuts[part], g_lo), b = cuts[part + 1];
    if (b <= a) continue;
    char* dst = slot + (slot_row + a - g_lo) * rb;
    const size_t bytes = static_cast<size_t>((b - a) * rb);
    if (part == 1) {
      CS_CUDA_TRY(cudaMemcpyAsync(dst, h_in + a * rb, bytes, cudaMemcpyHostToDevice, st));
    } else if (periodic) {
      const int64_t src = part == 0 ? a + ny : a - ny;
      CS_CUDA_TRY(cudaMemcpyAsync(dst, h_in + src * rb, bytes, cudaMemcpyHostToDevice, st));
    } else {
      CS_CUDA_TRY(cudaMemsetAsync(dst, 0, bytes, st));
    }
  }
  return CS_OK;
}

int compute_host_streamed(cs_plan* p, const void* h_in, void* h_out, cudaStream_t s) {
  const Stencil2DConfig& c = p->s2;
  int rc = ring_streams(p);
  if (rc != CS_OK) return rc;
  for (int k = 0; k < kRingSlots; ++k) {  // fresh copies: tile choice or FP64 mode may have changed
    p->ring_cfg[k] = c;
    p->ring_cfg[k].ny = p->ring_ny;
    p->ring_cfg[k].tmap_in = nullptr;
  }
  const int64_t ny = c.ny, nx = c.nx, eb = static_cast<int64_t>(p->elem_bytes), rb = nx * eb;
  const int64_t rows = p->ring_rows, nb = (ny + rows - 1) / rows;
  const bool periodic = c.bc == CS_BC_PERIODIC;
  // the rows and columns a sweep writes: all for periodic plans, the interior for non-periodic
  const int64_t w_lo = periodic ? 0 : c.top, w_hi = periodic ? ny : ny - c.bottom;
  const int64_t x_lo = periodic ? 0 : c.left, x_hi = periodic ? nx : nx - c.right;
  cudaStream_t sin = p->band_stream[0], sout = p->band_stream[1];
  cudaEvent_t* ev_in = p->band_event;
  cudaEvent_t* ev_comp = p->band_event + kRingSlots;
  cudaEvent_t* ev_out = p->band_event + 2 * kRingSlots;
  cudaEvent_t ev_start = p->band_event[3 * kRingSlots], ev_end = p->band_event[3 * kRingSlots + 1];
  const char* hi = static_cast<const char*>(h_in);
  char* ho = static_cast<char*>(h_out);
  CS_CUDA_TRY(cudaEventRecord(ev_start, s));
  CS_CUDA_TRY(cudaStreamWaitEvent(sin, ev_start, 0));
  CS_CUDA_TRY(cudaStreamWaitEvent(sout, ev_start, 0));
  for (int64_t b = 0; b < nb; ++b) {
    const int k = static_cast<int>(b % kRingSlots);
    const int64_t g0 = b * rows, g1 = std::min(ny, g0 + rows);
    // the rows the band's tiles stage: from g0 - top to the end of the last 64-row tile + bottom
    const int64_t r_lo = g0 - c.top, r_hi = (g1 + kStencilBandAlign - 1) / kStencilBandAlign * kStencilBandAlign + c.bottom;
    char* slot_in = static_cast<char*>(p->ring_in[k]);
    char* slot_out = static_cast<char*>(p->ring_out[k]);
    if (b >= kRingSlots) CS_CUDA_TRY(cudaStreamWaitEvent(sin, ev_comp[k], 0));  // slot's last sweep done
    rc = ring_fill(p, hi, slot_in, r_lo, r_hi, kRingTop - c.top, sin);
    if (rc != CS_OK) return rc;
    CS_CUDA_TRY(cudaEventRecord(ev_in[k], sin));
    CS_CUDA_TRY(cudaStreamWaitEvent(s, ev_in[k], 0));
    if (b >= kRingSlots) CS_CUDA_TRY(cudaStreamWaitEvent(s, ev_out[k], 0));  // slot's last copy-out done
    rc = stencil2d_launch_rows(&p->ring_cfg[k], slot_in, slot_out, kRingTop, kRingTop + (g1 - g0), s);
    if (rc != CS_OK) return rc;
    CS_CUDA_TRY(cudaEventRecord(ev_comp[k], s));
    CS_CUDA_TRY(cudaStreamWaitEvent(sout, ev_comp[k], 0));
    const int64_t o0 = std::max(g0, w_lo), o1 = std::min(g1, w_hi);
    if (o1 > o0 && x_hi > x_lo) {
      const char* src = slot_out + (kRingTop + o0 - g0) * rb + x_lo * eb;
      if (x_lo == 0 && x_hi == nx)
        CS_CUDA_TRY(cudaMemcpyAsync(ho + o0 * rb, src, static_cast<size_t>((o1 - o0) * rb), cudaMemcpyDeviceToHost, sout));
      else
        CS_CUDA_TRY(cudaMemcpy2DAsync(ho + o0 * rb + x_lo * eb, static_cast<size_t>(rb), src, static_cast<size_t>(rb),
                                      static_cast<size_t>((x_hi - x_lo) * eb), static_cast<size_t>(o1 - o0),
                                      cudaMemcpyDeviceToHost, sout));
    }
    CS_CUDA_TRY(cudaEventRecord(ev_out[k], sout));
  }
  CS_CUDA_TRY(cudaEventRecord(ev_end, sout));
  CS_CUDA_TRY(cudaStreamWaitEvent(s, ev_end, 0));
  CS_CUDA_TRY(cudaStreamSynchronize(s));
  return CS_OK;
}

bool is_2d(const cs_plan* p) { return p && (p->kind == kStencil2D || p->kind == kStencil2DHost); }

cs_plan* new_plan(int kind) {
  cs_plan* p = new (std::nothrow) cs_plan;
  if (!p) return nullptr;
  memset(p, 0, sizeof *p);
  p->kind = kind;
  return p;
}

}  // namespace

extern "C" {

const char* cs_last_error(void) { return cs::t_last_error.c_str(); }
int64_t cs_launch_count(void) { return cs::g_launches.load(); }
const char* cs_version(void) { return "custen_gb 0.1.0 sm_103a"; }

int cs_plan_create_2d(cs_plan_t* plan, const cs_stencil_desc* d, const void* d_in, void* d_out) {
  if (!plan) return set_error(CS_EINVAL, "null plan pointer");
  *plan = nullptr;
  int rc = validate_desc_common(d);
  if (rc != CS_OK) return rc;
  if (d->nx < 0 || d->ny < 0) return set_error(CS_EINVAL, "nx, ny must be >= 0");
  if (d->nx > (int64_t(1) << 40) / (d->ny > 0 ? d->ny : 1)) return set_error(CS_EINVAL, "grid too large");
  const size_t eb = d->dtype == CS_F32 ? 4 : 8;
  const int64_t elems = d->nx * d->ny;
  if (elems > 0 && (!d_in || !d_out)) return set_error(CS_EINVAL, "null device buffer");
  if (elems > 0 && (reinterpret_cast<uintptr_t>(d_in) % eb || reinterpret_cast<uintptr_t>(d_out) % eb))
    return set_error(CS_EINVAL, "buffers must be aligned to the element size");
  if (elems > 0 && overlaps(d_in, d_out, static_cast<size_t>(elems) * eb))
    return set_error(CS_EALIAS, "input and output buffers overlap (Sec. 2: outputs go to a separate buffer)");
  cs_plan* p = new_plan(kStencil2D);
  if (!p) return set_error(CS_ENOMEM, "out of host memory");
  rc = fill_2d_config(p, d);
  if (rc != CS_OK) { delete p; return rc; }
  p->d_in = d_in; p->d_out = d_out; p->elem_bytes = eb; p->elems = elems;
  *plan = p;
  return CS_OK;
}

int cs_plan_create_2d_host(cs_plan_t* plan, const cs_stencil_desc* d, int64_t device_bytes) {
  if (!plan) return set_error(CS_EINVAL, "null plan pointer");
  *plan = nullptr;
  int rc = validate_desc_common(d);
  if (rc != CS_OK) return rc;
  if (d->nx < 1 || d->ny < kRingMinRows)
    return set_error(CS_EINVAL, "a host-resident plan needs nx >= 1 and ny >= %lld", (long long)kRingMinRows);
  if (d->nx > (int64_t(1) << 40) / d->ny) return set_error(CS_EINVAL, "grid too large");
  if (device_bytes < 0) return set_error(CS_EINVAL, "device_bytes must be >= 0");
  const int64_t eb = d->dtype == CS_F32 ? 4 : 8;
  const int64_t budget = device_bytes ? device_bytes : (int64_t(512) << 20);
  // slots x (input + output) x (top + rows + bottom) rows of nx elements within the budget
  const int64_t row_pair = 2 * kRingSlots * d->nx * eb;
  int64_t rows = budget / row_pair - kRingTop - kRingBottom;
  rows = rows / kStencilBandAlign * kStencilBandAlign;
  const int64_t grid_rows = (d->ny + kStencilBandAlign - 1) / kStencilBandAlign * kStencilBandAlign;
  rows = std::min(rows, grid_rows);
  if (rows < kStencilBandAlign)
    return set_error(CS_EINVAL, "device_bytes %lld is below one %lld-row band per slot (%lld bytes)",
                     (long long)budget, (long long)kStencilBandAlign,
                     (long long)(row_pair * (kStencilBandAlign + kRingTop + kRingBottom)));
  cs_plan* p = new_plan(kStencil2DHost);
  if (!p) return set_error(CS_ENOMEM, "out of host memory");
  rc = fill_2d_config(p, d);
  if (rc != CS_OK) { delete p; return rc; }
  p->elem_bytes = static_cast<size_t>(eb);
  p->elems = d->nx * d->ny;
  p->ring_rows = rows;
  p->ring_ny = kRingTop + rows + kRingBottom;
  p->ring_cfg = new (std::nothrow) Stencil2DConfig[kRingSlots];
  const size_t slot_bytes = static_cast<size_t>(p->ring_ny * d->nx * eb);
  cudaError_t e = p->ring_cfg ? cudaSuccess : cudaErrorMemoryAllocation;
  for (int k = 0; k < kRingSlots && e == cudaSuccess; ++k) {
    e = cudaMalloc(&p->ring_in[k], slot_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&p->ring_out[k], slot_bytes);
  }
  if (e != cudaSuccess) {
    ring_free(p);
    stencil2d_release(&p->s2);
    delete p;
    return e == cudaErrorMemoryAllocation ? set_error(CS_ENOMEM, "band slots of %zu bytes: %s", slot_bytes, cudaGetErrorString(e))
                                          : cuda_error(e, "band slots");
  }
  p->ring_bytes = static_cast<int64_t>(2 * kRingSlots * slot_bytes);
  *plan = p;
  return CS_OK;
}

int cs_plan_create_weno_adv(cs_plan_t* plan, const cs_weno_desc* d, const void* d_c, const void* d_u,
                            const void* d_v, void* d_out) {
  if (!plan) return set_error(CS_EINVAL, "null plan pointer");
  *plan = nullptr;
  if (!d) return set_error(CS_EINVAL, "null WENO description");
  if (d->dtype != CS_F64 && d->dtype != CS_F32) return set_error(CS_EINVAL, "dtype must be CS_F64 or CS_F32");
  if (d->nx < 0 || d->ny < 0) return set_error(CS_EINVAL, "nx, ny must be >= 0");
  if (d->nx > (int64_t(1) << 40) / (d->ny > 0 ? d->ny : 1)) return set_error(CS_EINVAL, "grid too large");
  if (!(d->hx >= 1e-60 && d->hx <= 1e60 && d->hy >= 1e-60 && d->hy <= 1e60))
    return set_error(CS_EINVAL, "hx, hy must lie in [1e-60, 1e60]");
  const size_t eb = d->dtype == CS_F32 ? 4 : 8;
  const int64_t elems = d->nx * d->ny;
  if (elems > 0) {
    const void* f[4] = {d_c, d_u, d_v, d_out};
    for (const void* q : f) {
      if (!q) return set_error(CS_EINVAL, "null device buffer");
      if (reinterpret_cast<uintptr_t>(q) % eb) return set_error(CS_EINVAL, "buffers must be aligned to the element size");
    }
    const size_t bytes = static_cast<size_t>(elems) * eb;
    for (int i = 0; i < 3; ++i)
      if (overlaps(f[i], d_out, bytes))
        return set_error(CS_EALIAS, "the output must not overlap C, u or v (Sec. 2: blocks read overlapping halos)");
  }
  cs_plan* p = new_plan(kWeno);
  if (!p) return set_error(CS_ENOMEM, "out of host memory");
  p->weno.nx = d->nx;
  p->weno.ny = d->ny;
  p->weno.dtype = d->dtype;
  p->weno.hx = d->hx;
  p->weno.hy = d->hy;
  p->d_in = d_c; p->d_u = d_u; p->d_v = d_v; p->d_out = d_out;
  p->elem_bytes = eb;
  p->elems = elems;
  *plan = p;
  return CS_OK;
}

int cs_plan_host_info(cs_plan_t p, int64_t* band_rows, int64_t* device_bytes) {
  if (!p || p->kind != kStencil2DHost) return set_error(CS_EINVAL, "not a host-resident 2D plan");
  if (band_rows) *band_rows = p->ring_rows;
  if (device_bytes) *device_bytes = p->ring_bytes;
  return CS_OK;
}

int cs_plan_create_1d_batch(cs_plan_t* plan, const cs_stencil_desc* d, int64_t num_lines,
                            const int64_t* d_offsets, int64_t total_len, const void* d_in, void* d_out) {
  if (!plan) return set_error(CS_EINVAL, "null plan pointer");
  *plan = nullptr;
  int rc = validate_desc_common(d);
  if (rc != CS_OK) return rc;
  if (d->dir != CS_DIR_X || d->fn != CS_FN_NONE)
    return set_error(CS_EINVAL, "batched 1D lines take a weighted X stencil");
  if (num_lines < 0 || total_len < 0 || total_len > (int64_t(1) << 40))
    return set_error(CS_EINVAL, "num_lines, total_len out of range");
  if (num_lines > 0x7fffffff) return set_error(CS_EINVAL, "at most 2^31-1 lines");
  if (total_len > 0 && num_lines == 0) return set_error(CS_EINVAL, "elements without lines");
  if (!d_offsets) return set_error(CS_EINVAL, "null offsets");
  const size_t eb = d->dtype == CS_F32 ? 4 : 8;
  if (total_len > 0 && (!d_in || !d_out)) return set_error(CS_EINVAL, "null device buffer");
  if (total_len > 0 && (reinterpret_cast<uintptr_t>(d_in) % eb || reinterpret_cast<uintptr_t>(d_out) % eb))
    return set_error(CS_EINVAL, "buffers must be aligned to the element size");
  if (total_len > 0 && overlaps(d_in, d_out, static_cast<size_t>(total_len) * eb))
    return set_error(CS_EALIAS, "input and output buffers overlap");
  // offsets must be consistent: offsets[0] == 0, offsets[num_lines] == total_len, non-decreasing
  {
    std::vector<int64_t> h(static_cast<size_t>(num_lines) + 1);
    CS_CUDA_TRY(cudaMemcpy(h.data(), d_offsets, h.size() * sizeof(int64_t), cudaMemcpyDeviceToHost));
    if (h[0] != 0 || h[num_lines] != total_len)
      return set_error(CS_EINVAL, "offsets must start at 0 and end at total_len");
    for (int64_t m = 0; m < num_lines; ++m)
      if (h[m + 1] < h[m]) return set_error(CS_EINVAL, "offsets must be non-decreasing (line %lld)", (long long)m);
      else if (h[m + 1] - h[m] > 0x7fffffff) return set_error(CS_EINVAL, "line %lld is longer than 2^31-1", (long long)m);
  }
  cs_plan* p = new_plan(kBatch1D);
  if (!p) return set_error(CS_ENOMEM, "out of host memory");
  Batch1DConfig& c = p->b1;
  c.num_lines = num_lines; c.total_len = total_len; c.bc = d->bc; c.dtype = d->dtype;
  c.left = d->left; c.right = d->right;
  memcpy(c.weights, d->weights, sizeof(double) * (d->left + d->right + 1));
  c.d_offsets = d_offsets;
  rc = batch1d_prepare(&c, nullptr);
  if (rc == CS_OK) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = cuda_error(e, "building the line table");
  }
  if (rc != CS_OK) { batch1d_release(&c); delete p; return rc; }
  p->d_in = d_in; p->d_out = d_out; p->elem_bytes = eb; p->elems = total_len;
  *plan = p;
  return CS_OK;
}

int cs_compute(cs_plan_t p, void* stream) {
  if (!p) return set_error(CS_EINVAL, "null plan");
  if (p->kind == kCahnHilliard) return set_error(CS_EINVAL, "use cs_ch_step for a Cahn-Hilliard plan");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!p->use_graph) return launch_direct(p, s);
  if (!p->exec) {
    // capture on a private stream (the caller's may be the legacy stream, which cannot capture)
    cudaStream_t cap;
    CS_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    int64_t before = cs_launch_count();
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    int rc = e == cudaSuccess ? launch_direct(p, cap) : cuda_error(e, "cudaStreamBeginCapture");
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (rc != CS_OK) { if (g) cudaGraphDestroy(g); return rc; }
    if (e2 != cudaSuccess) return cuda_error(e2, "cudaStreamEndCapture");
    // capture does not launch: undo the count and remember how many kernels one replay runs
    p->graph_kernels = static_cast<int>(cs_launch_count() - before);
    count_launches(-p->graph_kernels);
    cudaError_t e3 = cudaGraphInstantiate(&p->exec, g, 0);
    if (e3 != cudaSuccess) { cudaGraphDestroy(g); p->exec = nullptr; return cuda_error(e3, "cudaGraphInstantiate"); }
    p->graph = g;
  }
  CS_CUDA_TRY(cudaGraphLaunch(p->exec, s));
  count_launches(p->graph_kernels);
  return CS_OK;
}

int cs_compute_group(const cs_plan_t* plans, int32_t count, void* stream) {
  if (count < 0 || (count > 0 && !plans)) return set_error(CS_EINVAL, "cs_compute_group: bad plan array");
  if (count == 0) return CS_OK;
  const cs_plan* first = plans[0];
  for (int32_t i = 0; i < count; ++i) {
    const cs_plan* p = plans[i];
    if (!p || p->kind != kStencil2D) return set_error(CS_EINVAL, "cs_compute_group: plan %d is not a 2D stencil plan", i);
    if (p->s2.variant < 0) return set_error(CS_EUNSUPPORTED, "cs_compute_group: plan %d uses the generic kernel", i);
    if (p->s2.dtype != first->s2.dtype || p->s2.variant != first->s2.variant || p->s2.tile_rows != first->s2.tile_rows)
      return set_error(CS_EINVAL, "cs_compute_group: plans must share dtype, stencil shape and tile shape");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int32_t b = 0; b < count; b += kMaxGroupJobs) {
    const int n = count - b < kMaxGroupJobs ? count - b : kMaxGroupJobs;
    const Stencil2DConfig* cfgs[kMaxGroupJobs];
    const void* ins[kMaxGroupJobs];
    void* outs[kMaxGroupJobs];
    for (int j = 0; j < n; ++j) {
      cfgs[j] = &plans[b + j]->s2;
      ins[j] = plans[b + j]->d_in;
      outs[j] = plans[b + j]->d_out;
    }
    int rc = stencil2d_group(cfgs, ins, outs, n, s);
    if (rc != CS_OK) return rc;
  }
  return CS_OK;
}

int cs_compute_host(cs_plan_t p, const void* h_in, void* h_out, void* stream) {
  if (!p) return set_error(CS_EINVAL, "null plan");
  if (p->kind == kWeno) return set_error(CS_EINVAL, "a WENO plan computes on device buffers (cs_compute)");
  if (p->kind == kCahnHilliard) return set_error(CS_EINVAL, "use cs_ch_step for a Cahn-Hilliard plan");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p->kind == kStencil2DHost) {
    if (!h_in || !h_out) return set_error(CS_EINVAL, "a host-resident plan needs both host buffers");
    if (overlaps(h_in, h_out, static_cast<size_t>(p->elems) * p->elem_bytes))
      return set_error(CS_EALIAS, "input and output buffers overlap");
    int rc = compute_host_streamed(p, h_in, h_out, s);
    return rc != CS_OK ? rc : stencil2d_check(&p->s2, s);
  }
  const size_t bytes = static_cast<size_t>(p->elems) * p->elem_bytes;
  if (p->kind == kStencil2D && h_in && h_out && bytes >= kBandMinBytes && p->s2.ny >= 2 * kStencilBandAlign) {
    int rc = compute_host_banded(p, h_in, h_out, s);
    return rc != CS_OK ? rc : stencil2d_check(&p->s2, s);
  }
  if (h_in && bytes) CS_CUDA_TRY(cudaMemcpyAsync(const_cast<void*>(p->d_in), h_in, bytes, cudaMemcpyHostToDevice, s));
  int rc = cs_compute(p, stream);
  if (rc != CS_OK) return rc;
  if (h_out && bytes) {
    CS_CUDA_TRY(cudaMemcpyAsync(h_out, p->d_out, bytes, cudaMemcpyDeviceToHost, s));
    CS_CUDA_TRY(cudaStreamSynchronize(s));
    if (p->kind == kStencil2D) return stencil2d_check(&p->s2, s);
  }
  return CS_OK;
}

int cs_plan_check(cs_plan_t p, void* stream) {
  if (!p) return set_error(CS_EINVAL, "null plan");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p->kind == kStencil2D || p->kind == kStencil2DHost) return stencil2d_check(&p->s2, s);
  CS_CUDA_TRY(cudaStreamSynchronize(s));
  return CS_OK;
}

int cs_plan_debug_stall(cs_plan_t p, int32_t tile) {
  if (!p || p->kind != kStencil2D) return set_error(CS_EINVAL, "not a 2D stencil plan on device buffers");
  p->s2.stall_from = tile < 0 ? -1 : tile;
  drop_graph(p);
  return CS_OK;
}

int cs_swap(cs_plan_t p) {
  if (!p) return set_error(CS_EINVAL, "null plan");
  if (p->kind == kCahnHilliard) return set_error(CS_EINVAL, "Cahn-Hilliard plans rotate their fields themselves");
  if (p->kind == kStencil2DHost) return set_error(CS_EINVAL, "a host-resident plan binds no device buffers");
  if (p->kind == kWeno) return set_error(CS_EINVAL, "a WENO plan's output is the advection term, not a new field");
  const void* in = p->d_in;
  p->d_in = p->d_out;
  p->d_out = const_cast<void*>(in);
  drop_graph(p);
  return CS_OK;
}

int cs_set_buffers(cs_plan_t p, const void* d_in, void* d_out) {
  if (!p) return set_error(CS_EINVAL, "null plan");
  if (p->kind == kCahnHilliard || p->kind == kStencil2DHost || p->kind == kWeno)
    return set_error(CS_EINVAL, "not a single-input device-buffer stencil plan");
  const size_t bytes = static_cast<size_t>(p->elems) * p->elem_bytes;
  if (bytes && (!d_in || !d_out)) return set_error(CS_EINVAL, "null device buffer");
  if (bytes && (reinterpret_cast<uintptr_t>(d_in) % p->elem_bytes || reinterpret_cast<uintptr_t>(d_out) % p->elem_bytes))
    return set_error(CS_EINVAL, "buffers must be aligned to the element size");
  if (bytes && overlaps(d_in, d_out, bytes)) return set_error(CS_EALIAS, "input and output buffers overlap");
  p->d_in = d_in;
  p->d_out = d_out;
  drop_graph(p);
  return CS_OK;
}

int cs_plan_set_fp64_mode(cs_plan_t p, int32_t mode) {
  if (!is_2d(p)) return set_error(CS_EINVAL, "not a 2D stencil plan");
  if (mode != CS_FP64_AUTO && mode != CS_FP64_NATIVE) return set_error(CS_EINVAL, "unknown FP64 mode %d", mode);
  p->s2.fp64_mode = mode;
  drop_graph(p);
  return CS_OK;
}

int cs_plan_set_tile_choice(cs_plan_t p, int32_t choice) {
  if (!is_2d(p)) return set_error(CS_EINVAL, "not a 2D stencil plan");
  if (choice < 0 || choice >= stencil2d_num_tile_choices()) return set_error(CS_EINVAL, "tile choice %d out of range", choice);
  stencil2d_set_tile_choice(&p->s2, choice);
  drop_graph(p);
  return CS_OK;
}

int cs_plan_get_tile_choice(cs_plan_t p, int32_t* choice) {
  if (!is_2d(p) || !choice) return set_error(CS_EINVAL, "not a 2D stencil plan");
  *choice = p->s2.use_tma ? 2 : (p->s2.tile_rows == 32 ? 0 : 1);
  return CS_OK;
}

int cs_plan_use_graph(cs_plan_t p, int enable) {
  if (!p) return set_error(CS_EINVAL, "null plan");
  if (p->kind == kCahnHilliard || p->kind == kStencil2DHost)
    return set_error(CS_EUNSUPPORTED, "graph replay is for device-buffer stencil plans");
  p->use_graph = enable != 0;
  if (!p->use_graph) drop_graph(p);
  return CS_OK;
}

int cs_autotune(cs_plan_t p, void* stream) {
  if (!p) return set_error(CS_EINVAL, "null plan");
  if (p->kind == kCahnHilliard) return ch_autotune(p->ch, static_cast<cudaStream_t>(stream));
  if (p->kind == kStencil2DHost || p->kind == kWeno) return CS_OK;  // one launch shape: nothing to choose
  if (p->elems == 0) return CS_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nchoices = p->kind == kStencil2D ? stencil2d_num_tile_choices() : batch1d_num_choices();
  cudaEvent_t e0, e1;
  CS_CUDA_TRY(cudaEventCreate(&e0));
  CS_CUDA_TRY(cudaEventCreate(&e1));
  int best = -1;
  float best_ms = 1e30f;
  int rc = CS_OK;
  const int reps = 3;
  for (int c = 0; c < nchoices && rc == CS_OK; ++c) {
    if (p->kind == kStencil2D) stencil2d_set_tile_choice(&p->s2, c);
    else p->b1.choice = c;
    rc = launch_direct(p, s);  // warm-up
    if (rc == CS_EUNSUPPORTED) {  // this candidate cannot run on this device: skip it
      rc = CS_OK;
      continue;
    }
    if (rc != CS_OK) break;
    float total = 0.f;
    for (int r = 0; r < reps && rc == CS_OK; ++r) {
      rc = cs::autotune_detail::flush_l2(s);  // time every launch from a cold L2
      if (rc != CS_OK) break;
      cudaEventRecord(e0, s);
      rc = launch_direct(p, s);
      cudaEventRecord(e1, s);
      cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) { rc = cuda_error(e, "autotune timing"); break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      total += ms;
    }
    if (rc == CS_OK && total < best_ms) { best_ms = total; best = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != CS_OK) return rc;
  if (best < 0) return set_error(CS_EUNSUPPORTED, "no launch shape of this plan runs on this device");
  if (p->kind == kStencil2D) {
    stencil2d_set_tile_choice(&p->s2, best);
    tune_store(stencil2d_shape_key(&p->s2), best);
  } else {
    p->b1.choice = best;
    tune_store(batch1d_shape_key(&p->b1), best);
  }
  drop_graph(p);
  return CS_OK;
}

int cs_destroy(cs_plan_t p) {
  if (!p) return CS_OK;
  drop_graph(p);
  if (p->band_ready) {
    for (auto& e : p->band_event) cudaEventDestroy(e);
    for (int i = 0; i < 2; ++i) cudaStreamDestroy(p->band_stream[i]);
  }
  if (p->kind == kStencil2DHost) ring_free(p);
  if (p->kind == kStencil2D || p->kind == kStencil2DHost) stencil2d_release(&p->s2);
  if (p->kind == kBatch1D) batch1d_release(&p->b1);
  if (p->kind == kCahnHilliard) ch_destroy(p->ch);
  if (p->kind == kCHBand) ch_band_destroy(p->chb);
  delete p;
  return CS_OK;
}

int cs_ch_create(cs_plan_t* plan, const cs_ch_desc* d, void* prev, void* cur, void* next) {
  if (!plan) return set_error(CS_EINVAL, "null plan pointer");
  *plan = nullptr;
  cs_plan* p = new_plan(kCahnHilliard);
  if (!p) return set_error(CS_ENOMEM, "out of host memory");
  int rc = ch_create(&p->ch, d, prev, cur, next);
  if (rc != CS_OK) { delete p; return rc; }
  *plan = p;
  return CS_OK;
}

int cs_ch_band_create(cs_plan_t* plan, const cs_ch_desc* d, int64_t rows) {
  if (!plan) return set_error(CS_EINVAL, "null plan pointer");
  *plan = nullptr;
  cs_plan* p = new_plan(kCHBand);
  if (!p) return set_error(CS_ENOMEM, "out of host memory");
  int rc = ch_band_create(&p->chb, d, rows);
  if (rc != CS_OK) { delete p; return rc; }
  *plan = p;
  return CS_OK;
}

int cs_ch_band_rhs(cs_plan_t p, const void* d_prev, const void* d_cur, double* d_rhs, double* d_sums, void* stream) {
  if (!p || p->kind != kCHBand) return set_error(CS_EINVAL, "not a Cahn-Hilliard band plan");
  return ch_band_rhs(p->chb, d_prev, d_cur, d_rhs, d_sums, static_cast<cudaStream_t>(stream));
}

int cs_ch_band_solve(cs_plan_t p, const double* d_in, double* d_out, void* stream) {
  if (!p || p->kind != kCHBand) return set_error(CS_EINVAL, "not a Cahn-Hilliard band plan");
  return ch_band_solve(p->chb, d_in, d_out, static_cast<cudaStream_t>(stream));
}

int cs_ch_band_update(cs_plan_t p, const void* d_prev, const void* d_cur, const double* d_v, void* d_next,
                      void* stream) {
  if (!p || p->kind != kCHBand) return set_error(CS_EINVAL, "not a Cahn-Hilliard band plan");
  return ch_band_update(p->chb, d_prev, d_cur, d_v, d_next, static_cast<cudaStream_t>(stream));
}

int cs_ch_partition(const cs_ch_desc* d, int32_t* chunks, int32_t* chunk_len) {
  return ch_partition(d, chunks, chunk_len);
}

int cs_ch_band_ycols_local(cs_plan_t p, int64_t chunk0, const double* d_in, double* d_ends, void* stream) {
  if (!p || p->kind != kCHBand) return set_error(CS_EINVAL, "not a Cahn-Hilliard band plan");
  return ch_band_ycols_local(p->chb, chunk0, d_in, d_ends, static_cast<cudaStream_t>(stream));
}

int cs_ch_band_ycols_correct(cs_plan_t p, int64_t chunk0, const double* d_ends_all, double* d_v, void* stream) {
  if (!p || p->kind != kCHBand) return set_error(CS_EINVAL, "not a Cahn-Hilliard band plan");
  return ch_band_ycols_correct(p->chb, chunk0, d_ends_all, d_v, static_cast<cudaStream_t>(stream));
}

int cs_ch_step(cs_plan_t p, int64_t nsteps, double* h_mass, double* h_energy, void* stream) {
  if (!p || p->kind != kCahnHilliard) return set_error(CS_EINVAL, "not a Cahn-Hilliard plan");
  return ch_step(p->ch, nsteps, h_mass, h_energy, static_cast<cudaStream_t>(stream));
}

int cs_ch_invariants(cs_plan_t p, double* mass, double* energy, void* stream) {
  if (!p || p->kind != kCahnHilliard) return set_error(CS_EINVAL, "not a Cahn-Hilliard plan");
  return ch_invariants(p->ch, mass, energy, static_cast<cudaStream_t>(stream));
}

int cs_ch_coarsening(cs_plan_t p, double* s, double* k1, void* stream) {
  if (!p || p->kind != kCahnHilliard) return set_error(CS_EINVAL, "not a Cahn-Hilliard plan");
  return ch_coarsening(p->ch, s, k1, static_cast<cudaStream_t>(stream));
}

int cs_ch_fields(cs_plan_t p, void** prev, void** cur, int64_t* steps) {
  if (!p || p->kind != kCahnHilliard) return set_error(CS_EINVAL, "not a Cahn-Hilliard plan");
  return ch_fields(p->ch, prev, cur, steps);
}

int cs_ch_set_fields(cs_plan_t p, void* prev, void* cur, void* next) {
  if (!p || p->kind != kCahnHilliard) return set_error(CS_EINVAL, "not a Cahn-Hilliard plan");
  return ch_set_fields(p->ch, prev, cur, next);
}

int cs_ch_solver_check(int64_t n, int32_t chunks, double a, int32_t boundary, double* residual) {
  if (boundary != CS_CH_PERIODIC && boundary != CS_CH_NOFLUX) return set_error(CS_EINVAL, "unknown boundary %d", boundary);
  return ch_solver_check(n, chunks, a, boundary == CS_CH_NOFLUX, residual);
}

int cs_ch_config(cs_plan_t p, int32_t* chunks, int32_t* chunk_len) {
  if (!p || p->kind != kCahnHilliard) return set_error(CS_EINVAL, "not a Cahn-Hilliard plan");
  return ch_config(p->ch, chunks, chunk_len);
}

}  // extern "C"
