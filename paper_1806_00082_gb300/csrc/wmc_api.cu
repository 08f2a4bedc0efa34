// Host side of the libwmc C ABI: argument checks, workspace layout, the
// per-step call sequence and its CUDA-graph capture.
#include <math.h>
#include <string.h>

#include <atomic>
#include <mutex>

#include <cuda.h>  // driver types only: the two driver calls below come through cudaGetDriverEntryPointByVersion

#include "wmc_internal.cuh"

namespace wmc {

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool params_ok(const wmc_params* p) {
  if (!p) return false;
  if (p->n_x < 1 || p->n_x > (1 << 24)) return false;
  if (p->Q < 2 || p->Q > 4096 || (p->Q & 1)) return false;
  if (p->n_M < 2 || p->n_M > 4096 || (p->n_M & 1)) return false;
  if (!(p->dx_m > 0) || !(p->mass_kg > 0) || !(p->dt_s > 0)) return false;
  if (p->bc_potential != 0 && p->bc_potential != 1) return false;
  if (p->child_wrap != 0 && p->child_wrap != 1) return false;
  // a particle may move at most to the neighbouring cell in one step
  const double d1 = ((kHbarJs * kPi) * p->dt_s) / ((p->mass_kg * (double)p->Q) * (p->dx_m * p->dx_m));
  const float dmax = (float)((double)(p->n_M / 2) * d1);
  if (!(dmax < 1.0f)) return false;
  return true;
}

Layout layout(const wmc_params& p) {
  Layout L;
  const size_t nx = (size_t)p.n_x, nM = (size_t)p.n_M;
  L.h = p.Q / 2;
  L.Kp = ((L.h - 1 + 31) / 32) * 32;
  if (L.Kp == 0) L.Kp = 32;
  L.Np = ((L.h + 63) / 64) * 64;
  L.Kp2 = ((L.h + 31) / 32) * 32;
  size_t o = 0;
  L.header = o; o = align256(o + sizeof(DevHeader));
  L.T = o; o = align256(o + sizeof(unsigned long long) * nx);
  L.R = o; o = align256(o + sizeof(unsigned long long) * (nx + 1));
  L.IP = o; o = align256(o + sizeof(int) * (nx + 1));
  L.reach = o; o = align256(o + nx);
  L.occ = o; o = align256(o + sizeof(int) * nx);
  L.row_map = o; o = align256(o + sizeof(int) * nx);
  L.VWh = o; o = align256(o + sizeof(float) * nx * (size_t)L.h);
  L.ccdf = o; o = align256(o + sizeof(long long) * nx * kCdfBlocks);
  L.scale = o; o = align256(o + sizeof(int) * nx);
  L.gamma = o; o = align256(o + sizeof(double) * nx);
  L.gthr = o; o = align256(o + sizeof(unsigned long long) * nx);
  L.thr_cell = o; o = align256(o + sizeof(unsigned long long) * nx);
  L.D = o; o = align256(o + sizeof(float) * nM);
  L.xlo = o; o = align256(o + sizeof(uint32_t) * nM);
  L.xhi = o; o = align256(o + sizeof(uint32_t) * nM);
  L.max_items = kMaxItemsBase + 2 * (long long)nx;
  L.items = o; o = align256(o + sizeof(int2) * (size_t)L.max_items);
  // pair queue: one entry per created pair of a step (events beyond it are
  // processed inside the step kernel instead)
  {
    const size_t want = nx * nM / 8;
    L.pair_cap = (unsigned)(want < (1u << 16) ? (1u << 16) : (want > (1u << 21) ? (1u << 21) : want));
  }
  L.pairs = o; o = align256(o + sizeof(uint4) * (size_t)L.pair_cap);
  L.B = o; o = align256(o + sizeof(float) * (size_t)L.Kp * (size_t)L.Np);
  L.B2 = o; o = align256(o + sizeof(float) * (size_t)L.Kp2 * (size_t)L.Np);
  L.tc = o; o = align256(o + tc_images_bytes(p));
  L.plan = o; o = align256(o + sizeof(PlanStatus) * ((nx + kPlanCells - 1) / kPlanCells));
  L.dft = o; o = align256(o + sizeof(double) * 2 * (size_t)p.Q);
  L.total = o;
  return L;
}

View view(const wmc_params& p, void* ws) {
  const Layout L = layout(p);
  char* b = static_cast<char*>(ws);
  View v;
  v.hdr = reinterpret_cast<DevHeader*>(b + L.header);
  v.T = reinterpret_cast<unsigned long long*>(b + L.T);
  v.R = reinterpret_cast<unsigned long long*>(b + L.R);
  v.IP = reinterpret_cast<int*>(b + L.IP);
  v.reach = reinterpret_cast<unsigned char*>(b + L.reach);
  v.occ = reinterpret_cast<int*>(b + L.occ);
  v.row_map = reinterpret_cast<int*>(b + L.row_map);
  v.VWh = reinterpret_cast<float*>(b + L.VWh);
  v.ccdf = reinterpret_cast<long long*>(b + L.ccdf);
  v.scale = reinterpret_cast<int*>(b + L.scale);
  v.gamma = reinterpret_cast<double*>(b + L.gamma);
  v.gthr = reinterpret_cast<unsigned long long*>(b + L.gthr);
  v.D = reinterpret_cast<float*>(b + L.D);
  v.xlo = reinterpret_cast<uint32_t*>(b + L.xlo);
  v.xhi = reinterpret_cast<uint32_t*>(b + L.xhi);
  v.thr_cell = reinterpret_cast<unsigned long long*>(b + L.thr_cell);
  v.items = reinterpret_cast<int2*>(b + L.items);
  v.pairs = reinterpret_cast<uint4*>(b + L.pairs);
  v.B = reinterpret_cast<float*>(b + L.B);
  v.B2 = reinterpret_cast<float*>(b + L.B2);
  v.tc = b + L.tc;
  v.plan = reinterpret_cast<PlanStatus*>(b + L.plan);
  v.dft = reinterpret_cast<double*>(b + L.dft);
  return v;
}

int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cached[dev]) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = n > 0 ? n : 1;
  }
  return cached[dev];
}

__global__ void k_set_step(DevHeader* hdr, uint32_t step) { hdr->step = step; }

__global__ void k_set_id_base(DevHeader* hdr, unsigned long long base) { hdr->id_base = base; }

__global__ void k_reset_counters(DevHeader* hdr) {
  hdr->particle_steps = 0;
  hdr->pairs = 0;
  hdr->absorbed = 0;
  hdr->absorbed_signed = 0;
  hdr->dropped = 0;
  hdr->dropped_signed = 0;
  hdr->flags = 0;
}

// One thread waits for *signal != 0 for at most max_cycles clock cycles (the
// bounded-wait pattern of the tensor-core kernels); giving up sets the
// timeout flag.
__global__ void k_check_wait(const uint32_t* signal, long long max_cycles, DevHeader* hdr) {
  const volatile uint32_t* sig = signal;
  const long long t0 = clock64();
  while (*sig == 0u) {
    if (clock64() - t0 > max_cycles) {
      atomicOr(&hdr->flags, WMC_FLAG_TIMEOUT);
      return;
    }
    __nanosleep(256);
  }
}

static wmc_status cuda_status(cudaError_t e) { return e == cudaSuccess ? WMC_OK : WMC_ERR_CUDA; }

static bool prec_supported(wmc_precision prec) {
  return prec == WMC_FP32 || prec == WMC_BF16 || prec == WMC_FP16 || prec == WMC_FP16_SPLIT || prec == WMC_TF32X3 ||
         prec == WMC_FP32_SIMT;
}

// the form that runs (internal code: WMC_FP32 = the CUDA cores)
static wmc_precision form_of(const wmc_params& p, wmc_precision prec, int net = 1, long long rows = 0) {
  return (wmc_precision)resolve_precision(p, (int)prec, net, rows);
}

// Kernel rows, CDFs and thresholds of the occupied list in the workspace:
// tensor-core contraction + CDF kernel for the reduced-precision forms; for
// FP32, fused for small windows, tiled contraction + CDF kernel otherwise.
static cudaError_t kernel_and_cdf_occupied(const wmc_params& p, const View& v, const float* V, wmc_precision prec,
                                           cudaStream_t s) {
  if (prec != WMC_FP32) {
    cudaError_t e = launch_kernel_eval_tc(p, (int)prec, V, v.occ, &v.hdr->n_occ, 0, p.n_x, v.tc, v.VWh,
                                          &v.hdr->flags, s);
    if (e != cudaSuccess) return e;
    return launch_cdf(p, v.VWh, &v.hdr->n_occ, 0, p.n_x, nullptr, v.gamma, v.scale, v.gthr, v.occ, v.thr_cell,
                      &v.hdr->flags, s, v.hdr, v.ccdf);
  }
  if (small_window(p))  // every cell a row, evaluated where the reach bits need it
    return launch_kernel_rows_small(p, V, nullptr, nullptr, p.n_x, p.n_x, v.B, v.VWh, v.ccdf, v.scale, v.gamma,
                                    v.gthr, v.thr_cell, &v.hdr->flags, s, v.reach, v.hdr);
  cudaError_t e = launch_kernel_eval(p, V, v.occ, &v.hdr->n_occ, 0, p.n_x, v.B, v.VWh, s);
  if (e != cudaSuccess) return e;
  return launch_cdf(p, v.VWh, &v.hdr->n_occ, 0, p.n_x, nullptr, v.gamma, v.scale, v.gthr, v.occ, v.thr_cell,
                    &v.hdr->flags, s, v.hdr, v.ccdf);
}

// Unique id of the calling thread's current CUDA context (0 if the driver
// cannot say).  Streams, events and graphs cached per device are kept with the
// id of the context that made them: after cudaDeviceReset the device has a
// new context and those handles are dropped (not destroyed: they died with
// their context) and made again.
static unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
    (void)cudaGetLastError();
  });
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_current && get_id && get_current(&c) == CUDA_SUCCESS && c && get_id(c, &id) == CUDA_SUCCESS) return id;
  return 0;
}

// Raises a kernel's dynamic shared-memory limit to at least `bytes`, calling
// the runtime only when the limit set before in this context is lower: the
// attribute persists, and a runtime call in front of every launch would sit
// between a caller's start event and the kernel.
cudaError_t raise_smem_limit(const void* func, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long ctx = current_context_id();
  struct Entry {
    const void* f;
    int dev;
    unsigned long long ctx;
    size_t bytes;
  };
  static std::mutex mu;
  static Entry table[256];
  static int n = 0;
  std::lock_guard<std::mutex> lock(mu);
  int slot = -1;
  for (int q = 0; q < n; ++q)
    if (table[q].f == func && table[q].dev == dev) {
      if (table[q].ctx == ctx && table[q].bytes >= bytes) return cudaSuccess;
      slot = q;
      break;
    }
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  if (slot < 0 && n < 256) slot = n++;
  if (slot >= 0) table[slot] = Entry{func, dev, ctx, bytes};
  return cudaSuccess;
}

// A second stream per device and a fork/join event pair, for running the
// single-block plan beside the kernel stage.
struct AuxStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  unsigned long long ctx = 0;
};

static bool aux_stream(AuxStream& out) {
  static std::mutex mu;
  static AuxStream per_dev[16];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) return false;
  const unsigned long long ctx = current_context_id();
  std::lock_guard<std::mutex> lock(mu);
  AuxStream& a = per_dev[dev];
  if (a.s && a.ctx != ctx) a = AuxStream();  // made in an earlier context of this device
  if (!a.s) {
    a.ctx = ctx;
    if (cudaStreamCreateWithFlags(&a.s, cudaStreamNonBlocking) != cudaSuccess) return false;
    if (cudaEventCreateWithFlags(&a.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&a.join, cudaEventDisableTiming) != cudaSuccess)
      return false;
  }
  out = a;
  return true;
}

// drift + kernel + step for one step, state in -> out, step number on the device
static wmc_status one_step(const wmc_params& p, const View& v, const float* V, const int32_t* in, int32_t* out,
                           wmc_precision prec, int device_step, uint32_t t, cudaStream_t s) {
  // the per-cell scan also zeroes the output histogram
  cudaError_t e;
  {
    NvtxRange r("wmc rebuild: per-cell scan");
    e = launch_rows(p, v, in, nullptr, s, out);
  }
  if (e != cudaSuccess) return WMC_ERR_CUDA;
  AuxStream aux;
  if (prec == WMC_FP32 && small_window(p) && aux_stream(aux)) {
    // the kernel stage needs only the reach bits, so the plan (ids, work items)
    // runs beside it on the second stream; the step waits for both
    if (cudaEventRecord(aux.fork, s) != cudaSuccess || cudaStreamWaitEvent(aux.s, aux.fork, 0) != cudaSuccess)
      return WMC_ERR_CUDA;
    {
      NvtxRange r("wmc rebuild: plan");
      e = launch_plan_scan(p, v, device_step, 0, aux.s);
    }
    if (e != cudaSuccess) return WMC_ERR_CUDA;
    if (cudaEventRecord(aux.join, aux.s) != cudaSuccess) return WMC_ERR_CUDA;
    {
      NvtxRange r("wmc kernel: rows, gamma, CDF");
      e = kernel_and_cdf_occupied(p, v, V, prec, s);
    }
    if (cudaStreamWaitEvent(s, aux.join, 0) != cudaSuccess || e != cudaSuccess) return WMC_ERR_CUDA;
  } else {
    {
      NvtxRange r("wmc rebuild: plan");
      e = launch_plan_scan(p, v, device_step, 1, s);
    }
    if (e != cudaSuccess) return WMC_ERR_CUDA;
    {
      NvtxRange r("wmc kernel: rows, gamma, CDF");
      e = kernel_and_cdf_occupied(p, v, V, prec, s);
    }
    if (e != cudaSuccess) return WMC_ERR_CUDA;
  }
  NvtxRange r("wmc step: drift, pairs, histogram");
  e = launch_step(p, v, in, t, device_step, out, s);
  return cuda_status(e);
}

// Events around the particle-step kernel, one pair per device, created on first
// use; `on` is read by every step launch, `recorded` once a pair has been
// enqueued (or captured) on that device.
struct StepTiming {
  std::mutex mu;
  std::atomic<int> on{0};
  cudaEvent_t ev[8][2] = {};
  bool recorded[8] = {};
  unsigned long long ctx[8] = {};
};
static StepTiming g_timing;

int step_timing_on() { return g_timing.on.load(); }

cudaError_t step_timing_record(cudaStream_t s, bool end) {
  if (!g_timing.on.load()) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 8) return cudaSuccess;  // devices beyond the table are not timed
  const unsigned long long ctx = current_context_id();
  std::lock_guard<std::mutex> lock(g_timing.mu);
  if (g_timing.ctx[dev] != ctx) {  // events of an earlier context of this device
    g_timing.ev[dev][0] = g_timing.ev[dev][1] = nullptr;
    g_timing.recorded[dev] = false;
    g_timing.ctx[dev] = ctx;
  }
  cudaEvent_t& ev = g_timing.ev[dev][end ? 1 : 0];
  if (!ev && (e = cudaEventCreate(&ev)) != cudaSuccess) return e;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if ((e = cudaStreamIsCapturing(s, &cs)) != cudaSuccess) return e;
  e = cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal)
                                          : cudaEventRecord(ev, s);
  if (e == cudaSuccess && end) g_timing.recorded[dev] = true;
  return e;
}

// Cached executable graphs of the step pair a -> b -> a (or of one step), one
// per configuration (parameters, buffers, workspace, precision, stream,
// device, step timing), for the last few configurations used: a caller that
// alternates between buffer sets (copies of the next state overlapping the
// current step) reuses its graphs instead of recapturing.
constexpr int kGraphSlots = 4;
struct GraphSlot {
  bool valid = false;
  unsigned long long last_use = 0;
  wmc_params p;
  const void *V, *a, *b, *ws;
  int prec;
  cudaStream_t stream;
  int device;
  unsigned long long ctx;
  int timing;
  cudaGraphExec_t exec = nullptr;
};
struct GraphCache {
  std::mutex mu;
  unsigned long long uses = 0;
  GraphSlot slot[kGraphSlots];
};
static GraphCache g_graph;   // the step pair a -> b -> a
static GraphCache g_graph1;  // one step a -> b and the copy back to a (odd step counts)

// Launches the cached graph of these arguments, capturing `body` into the
// least recently used slot first if no slot holds this configuration.
template <class Body>
static wmc_status launch_cached(GraphCache& gc, const wmc_params* p, const float* V, const int32_t* a,
                                const int32_t* b, const void* ws, wmc_precision prec, cudaStream_t s, int launches,
                                Body body) {
  std::lock_guard<std::mutex> lock(gc.mu);
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long ctx = current_context_id();
  const int timing = step_timing_on();
  GraphSlot* hit = nullptr;
  GraphSlot* victim = &gc.slot[0];
  for (GraphSlot& g : gc.slot) {
    if (g.valid && g.device == dev && g.ctx != ctx) {  // made in an earlier context of this device
      g.valid = false;
      g.exec = nullptr;
    }
    if (g.valid && memcmp(&g.p, p, sizeof(wmc_params)) == 0 && g.V == V && g.a == a && g.b == b && g.ws == ws &&
        g.prec == (int)prec && g.stream == s && g.device == dev && g.timing == timing) {
      hit = &g;
      break;
    }
    if (!g.valid || (victim->valid && g.last_use < victim->last_use)) victim = &g;
  }
  if (!hit) {
    GraphSlot& gs = *victim;
    if (gs.exec) {
      cudaGraphExecDestroy(gs.exec);
      gs.exec = nullptr;
    }
    gs.valid = false;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return WMC_ERR_CUDA;
    const wmc_status st = body();
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (st != WMC_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return st != WMC_OK ? st : WMC_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&gs.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return WMC_ERR_CUDA;
    gs.valid = true;
    gs.p = *p;
    gs.V = V;
    gs.a = a;
    gs.b = b;
    gs.ws = ws;
    gs.prec = (int)prec;
    gs.stream = s;
    gs.device = dev;
    gs.ctx = ctx;
    gs.timing = timing;
    hit = &gs;
  }
  hit->last_use = ++gc.uses;
  for (int q = 0; q < launches; ++q)
    if (cudaGraphLaunch(hit->exec, s) != cudaSuccess) return WMC_ERR_CUDA;
  return WMC_OK;
}

}  // namespace wmc

using namespace wmc;

extern "C" {

const char* wmc_version(void) { return "libwmc 0.1 (sm_103a)"; }

const char* wmc_status_string(wmc_status s) {
  switch (s) {
    case WMC_OK: return "ok";
    case WMC_ERR_ARG: return "invalid argument";
    case WMC_ERR_CAPACITY: return "capacity exceeded";
    case WMC_ERR_RATE: return "gamma dt >= 1";
    case WMC_ERR_CUDA: return "CUDA error";
    case WMC_ERR_TIMEOUT: return "device wait timed out";
    case WMC_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

size_t wmc_workspace_size(const wmc_params* p) {
  if (!params_ok(p)) return 0;
  return layout(*p).total;
}

wmc_status wmc_init(const wmc_params* p, void* ws, size_t ws_bytes, wmc_stream_t stream) {
  if (!params_ok(p) || !ws) return WMC_ERR_ARG;
  if (((uintptr_t)ws & 255) != 0) return WMC_ERR_ARG;
  const Layout L = layout(*p);
  if (ws_bytes < L.total) return WMC_ERR_ARG;
  const View v = view(*p, ws);
  (void)num_sms();
  prepare_step(*p);
  cudaError_t e = launch_init_tables(*p, v, (cudaStream_t)stream);
  if (e == cudaSuccess) e = launch_init_tc_images(*p, v.tc, (cudaStream_t)stream);
  return cuda_status(e);
}

wmc_status wmc_reset_counters(const wmc_params* p, void* ws, wmc_stream_t stream) {
  if (!params_ok(p) || !ws) return WMC_ERR_ARG;
  const View v = view(*p, ws);
  k_reset_counters<<<1, 1, 0, (cudaStream_t)stream>>>(v.hdr);
  return cuda_status(cudaGetLastError());
}

wmc_status wmc_check_wait(const wmc_params* p, const uint32_t* signal, uint64_t max_cycles, void* ws,
                          wmc_stream_t stream) {
  if (!params_ok(p) || !signal || !ws || max_cycles > (1ull << 34)) return WMC_ERR_ARG;
  const View v = view(*p, ws);
  k_check_wait<<<1, 1, 0, (cudaStream_t)stream>>>(signal, (long long)max_cycles, v.hdr);
  return cuda_status(cudaGetLastError());
}

wmc_status wmc_set_id_base(const wmc_params* p, void* ws, uint64_t id_base, wmc_stream_t stream) {
  if (!params_ok(p) || !ws || id_base >= (1ull << 32)) return WMC_ERR_ARG;
  const View v = view(*p, ws);
  k_set_id_base<<<1, 1, 0, (cudaStream_t)stream>>>(v.hdr, (unsigned long long)id_base);
  return cuda_status(cudaGetLastError());
}

wmc_status wmc_step_timing(int32_t enable) {
  g_timing.on.store(enable ? 1 : 0);
  return WMC_OK;
}

wmc_status wmc_step_timing_read(float* ms) {
  if (!ms) return WMC_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return WMC_ERR_CUDA;
  cudaEvent_t b = nullptr, e = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_timing.mu);
    if (dev < 0 || dev >= 8 || !g_timing.recorded[dev] || g_timing.ctx[dev] != current_context_id())
      return WMC_ERR_UNSUPPORTED;
    b = g_timing.ev[dev][0];
    e = g_timing.ev[dev][1];
  }
  if (cudaEventSynchronize(e) != cudaSuccess) return WMC_ERR_CUDA;
  return cudaEventElapsedTime(ms, b, e) == cudaSuccess ? WMC_OK : WMC_ERR_CUDA;
}

wmc_status wmc_get_counters(const wmc_params* p, const void* ws, wmc_counters* out, wmc_stream_t stream) {
  if (!params_ok(p) || !ws || !out) return WMC_ERR_ARG;
  DevHeader h;
  const View v = view(*p, const_cast<void*>(ws));
  cudaError_t e = cudaMemcpyAsync(&h, v.hdr, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return WMC_ERR_CUDA;
  out->population = h.population;
  out->particle_steps = h.particle_steps;
  out->pairs = h.pairs;
  out->absorbed = h.absorbed;
  out->absorbed_signed = h.absorbed_signed;
  out->dropped = h.dropped;
  out->dropped_signed = h.dropped_signed;
  out->n_occ = h.n_occ;
  out->n_items = h.n_items;
  out->flags = h.flags;
  out->step = h.step;
  if (h.magic != kMagic) return WMC_ERR_ARG;
  return WMC_OK;
}

wmc_status wmc_kernel_eval(const wmc_params* p, const float* V, const int32_t* occ, int32_t n_occ,
                           wmc_precision prec, float* VWh, void* ws, wmc_stream_t stream) {
  NvtxRange nvtx("wmc_kernel_eval");
  if (!params_ok(p) || !V || !ws || n_occ < 0 || (n_occ > 0 && (!occ || !VWh))) return WMC_ERR_ARG;
  if (!prec_supported(prec)) return WMC_ERR_UNSUPPORTED;
  if (n_occ == 0) return WMC_OK;
  const View v = view(*p, ws);
  prec = form_of(*p, prec, 1, n_occ);
  if (prec != WMC_FP32)
    return cuda_status(launch_kernel_eval_tc(*p, (int)prec, V, occ, nullptr, n_occ, n_occ, v.tc, VWh, &v.hdr->flags,
                                             (cudaStream_t)stream));
  if (small_window(*p))
    return cuda_status(launch_kernel_rows_small(*p, V, occ, nullptr, n_occ, n_occ, v.B, VWh, nullptr, nullptr,
                                                nullptr, nullptr, nullptr, nullptr, (cudaStream_t)stream));
  return cuda_status(launch_kernel_eval(*p, V, occ, nullptr, n_occ, n_occ, v.B, VWh, (cudaStream_t)stream));
}

wmc_status wmc_kernel_eval_n2(const wmc_params* p, const float* V, const int32_t* occ, int32_t n_occ,
                              wmc_precision prec, float* VWh, void* ws, wmc_stream_t stream) {
  NvtxRange nvtx("wmc_kernel_eval_n2");
  if (!params_ok(p) || !V || !ws || n_occ < 0 || (n_occ > 0 && (!occ || !VWh))) return WMC_ERR_ARG;
  if (!prec_supported(prec)) return WMC_ERR_UNSUPPORTED;
  if (prec == WMC_TF32X3) return WMC_ERR_UNSUPPORTED;
  if (n_occ == 0) return WMC_OK;
  prec = form_of(*p, prec, 2);
  const View v = view(*p, ws);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (prec != WMC_FP32)
    e = launch_kernel_eval_tc(*p, (int)prec, V, occ, nullptr, n_occ, n_occ, v.tc, VWh, &v.hdr->flags, s, 2);
  else if (small_window(*p))
    e = launch_kernel_rows_small(*p, V, occ, nullptr, n_occ, n_occ, v.B2, VWh, nullptr, nullptr, nullptr, nullptr,
                                 nullptr, nullptr, s, nullptr, nullptr, 2);
  else
    e = launch_kernel_eval(*p, V, occ, nullptr, n_occ, n_occ, v.B2, VWh, s, 2);
  if (e == cudaErrorNotSupported) return WMC_ERR_UNSUPPORTED;
  return cuda_status(e);
}

wmc_status wmc_kernel_eval_dft(const wmc_params* p, const float* V, float* VWh, void* ws, wmc_stream_t stream) {
  NvtxRange nvtx("wmc_kernel_eval_dft");
  if (!params_ok(p) || !V || !VWh || !ws) return WMC_ERR_ARG;
  const View v = view(*p, ws);
  return cuda_status(launch_kernel_dft(*p, V, v.dft, VWh, (cudaStream_t)stream));
}

wmc_status wmc_kernel_cdf(const wmc_params* p, const float* VWh, int32_t n_rows, int64_t* cdf, double* gamma,
                          int32_t* scale, wmc_stream_t stream) {
  if (!params_ok(p) || n_rows < 0 || (n_rows > 0 && (!VWh || !gamma))) return WMC_ERR_ARG;
  if (n_rows == 0) return WMC_OK;
  return cuda_status(launch_cdf(*p, VWh, nullptr, n_rows, n_rows, reinterpret_cast<long long*>(cdf), gamma, scale,
                                nullptr, nullptr, nullptr, nullptr, (cudaStream_t)stream));
}

wmc_status wmc_annihilate(const wmc_params* p, const int32_t* hist, int64_t* rho, void* ws, wmc_stream_t stream) {
  NvtxRange nvtx("wmc_annihilate");
  if (!params_ok(p) || !hist || !ws) return WMC_ERR_ARG;
  const View v = view(*p, ws);
  return cuda_status(launch_plan(*p, v, hist, rho, 0, (cudaStream_t)stream));
}

wmc_status wmc_kernel_eval_occupied(const wmc_params* p, const float* V, wmc_precision prec, void* ws,
                                    wmc_stream_t stream) {
  if (!params_ok(p) || !V || !ws) return WMC_ERR_ARG;
  if (!prec_supported(prec)) return WMC_ERR_UNSUPPORTED;
  const View v = view(*p, ws);
  return cuda_status(kernel_and_cdf_occupied(*p, v, V, form_of(*p, prec), (cudaStream_t)stream));
}

wmc_status wmc_kernel_table_occupied(const wmc_params* p, const float* table, void* ws, wmc_stream_t stream) {
  if (!params_ok(p) || !table || !ws) return WMC_ERR_ARG;
  const View v = view(*p, ws);
  const Layout L = layout(*p);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_gather_table(*p, table, v.occ, &v.hdr->n_occ, p->n_x, v.VWh, s);
  if (e == cudaSuccess)
    e = launch_cdf(*p, v.VWh, &v.hdr->n_occ, 0, p->n_x, nullptr, v.gamma, v.scale, v.gthr, v.occ, v.thr_cell,
                   &v.hdr->flags, s, v.hdr, v.ccdf);
  return cuda_status(e);
}

wmc_status wmc_step(const wmc_params* p, const int32_t* hist_in, uint32_t t, int32_t* hist_out, void* ws,
                    wmc_stream_t stream) {
  NvtxRange nvtx("wmc_step");
  if (!params_ok(p) || !hist_in || !hist_out || !ws || hist_in == hist_out || t == 0) return WMC_ERR_ARG;
  const View v = view(*p, ws);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(hist_out, 0, sizeof(int32_t) * (size_t)p->n_x * (size_t)p->n_M, s);
  if (e == cudaSuccess) e = launch_step(*p, v, hist_in, t, 0, hist_out, s);
  return cuda_status(e);
}

wmc_status wmc_run(const wmc_params* p, const float* V, int32_t* hist_a, int32_t* hist_b, uint32_t t_first,
                   int32_t n_steps, wmc_precision prec, int32_t use_graph, void* ws, wmc_stream_t stream) {
  NvtxRange nvtx("wmc_run");
  if (!params_ok(p) || !V || !hist_a || !hist_b || hist_a == hist_b || !ws || n_steps < 0 || t_first == 0)
    return WMC_ERR_ARG;
  if (!prec_supported(prec)) return WMC_ERR_UNSUPPORTED;
  if (n_steps == 0) return WMC_OK;
  prec = form_of(*p, prec);
  const View v = view(*p, ws);
  cudaStream_t s = (cudaStream_t)stream;
  k_set_step<<<1, 1, 0, s>>>(v.hdr, t_first - 1u);
  if (cudaGetLastError() != cudaSuccess) return WMC_ERR_CUDA;
  const int pairs = n_steps / 2;
  const size_t state_bytes = sizeof(int32_t) * (size_t)p->n_x * (size_t)p->n_M;
  // the odd last step: a -> b, then the state copied back to a
  auto odd_step = [&]() -> wmc_status {
    const wmc_status st = one_step(*p, v, V, hist_a, hist_b, prec, 1, 0, s);
    if (st != WMC_OK) return st;
    return cudaMemcpyAsync(hist_a, hist_b, state_bytes, cudaMemcpyDeviceToDevice, s) == cudaSuccess ? WMC_OK
                                                                                                   : WMC_ERR_CUDA;
  };
  if (use_graph && s != nullptr) {
    if (pairs > 0) {
      const wmc_status st = launch_cached(g_graph, p, V, hist_a, hist_b, ws, prec, s, pairs, [&]() -> wmc_status {
        const wmc_status st1 = one_step(*p, v, V, hist_a, hist_b, prec, 1, 0, s);
        return st1 == WMC_OK ? one_step(*p, v, V, hist_b, hist_a, prec, 1, 0, s) : st1;
      });
      if (st != WMC_OK) return st;
    }
    if (n_steps & 1) {
      const wmc_status st = launch_cached(g_graph1, p, V, hist_a, hist_b, ws, prec, s, 1, odd_step);
      if (st != WMC_OK) return st;
    }
    return WMC_OK;
  }
  for (int q = 0; q < pairs; ++q) {
    wmc_status st = one_step(*p, v, V, hist_a, hist_b, prec, 1, 0, s);
    if (st == WMC_OK) st = one_step(*p, v, V, hist_b, hist_a, prec, 1, 0, s);
    if (st != WMC_OK) return st;
  }
  if (n_steps & 1) return odd_step();
  return WMC_OK;
}

wmc_status wmc_density(const wmc_params* p, const int32_t* hist, int64_t* rho, wmc_stream_t stream) {
  if (!params_ok(p) || !hist || !rho) return WMC_ERR_ARG;
  return cuda_status(launch_density(*p, hist, rho, (cudaStream_t)stream));
}

wmc_status wmc_materialize(const wmc_params* p, const int32_t* hist, uint32_t t, int32_t* cell, float* f,
                           int16_t* M, int8_t* sign, int64_t capacity, void* ws, wmc_stream_t stream) {
  if (!params_ok(p) || !hist || !ws || capacity < 0) return WMC_ERR_ARG;
  if (capacity > 0 && (!cell || !f || !M || !sign)) return WMC_ERR_ARG;
  const View v = view(*p, ws);
  return cuda_status(launch_materialize(*p, v, hist, t, cell, f, M, sign, capacity, (cudaStream_t)stream));
}

wmc_status wmc_philox_throughput(uint32_t key0, uint32_t key1, int32_t pairs_per_thread, uint32_t* out,
                                 int64_t n_threads, wmc_stream_t stream) {
  if (!out || pairs_per_thread < 1 || n_threads < 256 || (n_threads % 256) != 0 || n_threads / 256 > 0x7fffffff)
    return WMC_ERR_ARG;
  if ((long long)pairs_per_thread * n_threads >= (1ll << 32)) return WMC_ERR_ARG;  // counters stay distinct
  return cuda_status(launch_philox_throughput(key0, key1, pairs_per_thread, out, n_threads, (cudaStream_t)stream));
}

wmc_status wmc_get_error(const wmc_params* p, const void* ws, wmc_stream_t stream, wmc_status* device_status,
                         char* msg, size_t len) {
  if (!params_ok(p) || !ws || !device_status) return WMC_ERR_ARG;
  wmc_counters c;
  const wmc_status st = wmc_get_counters(p, ws, &c, stream);
  if (st != WMC_OK) return st;
  wmc_status d = WMC_OK;
  const char* text = "no device condition";
  if (c.flags & WMC_FLAG_TIMEOUT) {
    d = WMC_ERR_TIMEOUT;
    text = "a bounded device wait gave up (WMC_FLAG_TIMEOUT)";
  } else if (c.flags & WMC_FLAG_CAPACITY) {
    d = WMC_ERR_CAPACITY;
    text = "population >= 2^32, work items or an output capacity exceeded (WMC_FLAG_CAPACITY)";
  } else if (c.flags & WMC_FLAG_RATE) {
    d = WMC_ERR_RATE;
    text = "gamma dt >= 1 in an evaluated cell (WMC_FLAG_RATE)";
  }
  *device_status = d;
  if (msg && len) {
    size_t n = strlen(text);
    if (n >= len) n = len - 1;
    memcpy(msg, text, n);
    msg[n] = '\0';
  }
  return WMC_OK;
}

wmc_status wmc_philox4x32_10(const uint32_t* ctr, uint32_t key0, uint32_t key1, int64_t n, uint32_t* out,
                             wmc_stream_t stream) {
  if (n < 0 || (n > 0 && (!ctr || !out))) return WMC_ERR_ARG;
  return cuda_status(launch_philox(ctr, key0, key1, n, out, (cudaStream_t)stream));
}

}  // extern "C"
