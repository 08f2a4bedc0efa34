// Batched form: many independent simulations of uneven size advanced together,
// one launch per phase for the whole batch (and the step pair captured in a
// CUDA graph).  Each simulation keeps its own parameters, potential, net
// histogram and Philox stream (counter word 3 = its sim index); its results
// are bit-identical to running it alone.
//
// Cells of all simulations are concatenated (global cell c = cell_off[s] + i);
// per-cell arrays (survivors, id prefix, reach bits, row map, thresholds) are
// indexed by global cell, and the survivor-id prefix, work items and occupied
// list come from one scan over all cells (three passes: block sums, a scan of
// the block sums, and the final block scan).  Ids restart at 0 in every
// simulation: id = G[c] - G[cell_off[s]] + (offset within the cell).
//
// The work-item size (threads x ids per thread) is a run-time parameter chosen
// by wmc_batch_autotune; the results do not depend on it.
#include <string.h>

#include <mutex>
#include <vector>

#include "wmc_device.cuh"

namespace wmc {

namespace {

struct SimDesc {
  int n_x, Q, n_M, bc, wrap, h, log2_nM, Kp, Np;
  uint32_t sim, k0, k1;
  float c;
  float pad;
  double dt, d1;
  long long cell_off, hist_off, tab_off, sine_off;
};

constexpr int kScanCells = 1024;  // cells per block of the batch scan
constexpr int kScanThreads = 256;
constexpr int kBatchMaxH = 128;   // warp-per-row kernel: Q <= 256
constexpr int kBatchRowWarps = 8;

struct BatchLayout {
  size_t header, descs, sim_base, cell_sim, T, G, reach, row_map, thr_cell, occ, items, blk, VWh, cdf, gamma, gthr,
      D, xlo, xhi, sine, total;
  long long n_cells, hist_elems, tab_elems, sine_elems, max_items;
  int n_blk, H, NM;
};

int ceil_log2_host(int n) {
  int L = 0;
  while ((1 << L) < n) ++L;
  return L;
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

bool batch_ok(const wmc_params* ps, int n) {
  if (!ps || n < 1 || n > (1 << 20)) return false;
  for (int s = 0; s < n; ++s) {
    if (!params_ok(&ps[s])) return false;
    if (ps[s].Q / 2 > kBatchMaxH) return false;
  }
  return true;
}

BatchLayout batch_layout(const wmc_params* ps, int n) {
  BatchLayout L;
  L.n_cells = 0;
  L.hist_elems = 0;
  L.tab_elems = 0;
  L.sine_elems = 0;
  L.H = 1;
  L.NM = 2;
  for (int s = 0; s < n; ++s) {
    const int h = ps[s].Q / 2;
    const int Kp = ((h - 1 + 31) / 32) * 32 > 0 ? ((h - 1 + 31) / 32) * 32 : 32;
    const int Np = ((h + 63) / 64) * 64;
    L.n_cells += ps[s].n_x;
    L.hist_elems += (long long)ps[s].n_x * ps[s].n_M;
    L.tab_elems += ps[s].n_M;
    L.sine_elems += (long long)Kp * Np;
    if (h > L.H) L.H = h;
    if (ps[s].n_M > L.NM) L.NM = ps[s].n_M;
  }
  L.n_blk = (int)((L.n_cells + kScanCells - 1) / kScanCells);
  L.max_items = 2 * L.n_cells + (1ll << 23);
  const size_t nc = (size_t)L.n_cells;
  size_t o = 0;
  L.header = o; o = al256(o + sizeof(DevHeader));
  L.descs = o; o = al256(o + sizeof(SimDesc) * n);
  L.sim_base = o; o = al256(o + sizeof(unsigned long long) * n);
  L.cell_sim = o; o = al256(o + sizeof(int) * nc);
  L.T = o; o = al256(o + sizeof(unsigned long long) * nc);
  L.G = o; o = al256(o + sizeof(unsigned long long) * (nc + 1));
  L.reach = o; o = al256(o + nc);
  L.row_map = o; o = al256(o + sizeof(int) * nc);
  L.thr_cell = o; o = al256(o + sizeof(unsigned long long) * nc);
  L.occ = o; o = al256(o + sizeof(int) * nc);
  L.items = o; o = al256(o + sizeof(int2) * (size_t)L.max_items);
  L.blk = o; o = al256(o + sizeof(unsigned long long) * 3 * (size_t)(L.n_blk + 1));
  L.VWh = o; o = al256(o + sizeof(float) * nc * (size_t)L.H);
  L.cdf = o; o = al256(o + sizeof(long long) * nc * (size_t)L.NM);
  L.gamma = o; o = al256(o + sizeof(double) * nc);
  L.gthr = o; o = al256(o + sizeof(unsigned long long) * nc);
  L.D = o; o = al256(o + sizeof(float) * (size_t)L.tab_elems);
  L.xlo = o; o = al256(o + sizeof(uint32_t) * (size_t)L.tab_elems);
  L.xhi = o; o = al256(o + sizeof(uint32_t) * (size_t)L.tab_elems);
  L.sine = o; o = al256(o + sizeof(float) * (size_t)L.sine_elems);
  L.total = o;
  return L;
}

struct BatchView {
  DevHeader* hdr;
  SimDesc* descs;
  unsigned long long *sim_base, *T, *G, *thr_cell, *gthr, *blk;
  int *cell_sim, *row_map, *occ;
  unsigned char* reach;
  int2* items;
  float *VWh, *D, *sine;
  long long* cdf;
  double* gamma;
  uint32_t *xlo, *xhi;
};

BatchView batch_view(const BatchLayout& L, void* ws) {
  char* b = static_cast<char*>(ws);
  BatchView v;
  v.hdr = reinterpret_cast<DevHeader*>(b + L.header);
  v.descs = reinterpret_cast<SimDesc*>(b + L.descs);
  v.sim_base = reinterpret_cast<unsigned long long*>(b + L.sim_base);
  v.cell_sim = reinterpret_cast<int*>(b + L.cell_sim);
  v.T = reinterpret_cast<unsigned long long*>(b + L.T);
  v.G = reinterpret_cast<unsigned long long*>(b + L.G);
  v.reach = reinterpret_cast<unsigned char*>(b + L.reach);
  v.row_map = reinterpret_cast<int*>(b + L.row_map);
  v.thr_cell = reinterpret_cast<unsigned long long*>(b + L.thr_cell);
  v.occ = reinterpret_cast<int*>(b + L.occ);
  v.items = reinterpret_cast<int2*>(b + L.items);
  v.blk = reinterpret_cast<unsigned long long*>(b + L.blk);
  v.VWh = reinterpret_cast<float*>(b + L.VWh);
  v.cdf = reinterpret_cast<long long*>(b + L.cdf);
  v.gamma = reinterpret_cast<double*>(b + L.gamma);
  v.gthr = reinterpret_cast<unsigned long long*>(b + L.gthr);
  v.D = reinterpret_cast<float*>(b + L.D);
  v.xlo = reinterpret_cast<uint32_t*>(b + L.xlo);
  v.xhi = reinterpret_cast<uint32_t*>(b + L.xhi);
  v.sine = reinterpret_cast<float*>(b + L.sine);
  return v;
}

// simulation owning element e of a concatenation with offsets off[0..n)
__device__ __forceinline__ int owner(const SimDesc* __restrict__ d, int n, long long e, int which) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    const long long o = which == 0 ? d[mid].cell_off : (which == 1 ? d[mid].tab_off : d[mid].sine_off);
    if (o <= e) lo = mid; else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------- set-up
__global__ void k_b_init(const SimDesc* __restrict__ d, int n, long long n_cells, long long tab_elems,
                         long long sine_elems, int* __restrict__ cell_sim, float* __restrict__ D,
                         uint32_t* __restrict__ xlo, uint32_t* __restrict__ xhi, float* __restrict__ sine,
                         DevHeader* hdr) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nt = (long long)gridDim.x * blockDim.x;
  if (tid == 0) {
    DevHeader z = {};
    z.magic = kMagic;
    *hdr = z;
  }
  for (long long c = tid; c < n_cells; c += nt) cell_sim[c] = owner(d, n, c, 0);
  for (long long e = tid; e < tab_elems; e += nt) {
    const SimDesc& s = d[owner(d, n, e, 1)];
    const int k = (int)(e - s.tab_off);
    const float dd = __double2float_rn((double)(k - s.n_M / 2) * s.d1);
    D[e] = dd;
    uint32_t lo = 0u, hi = 0xffffffffu;
    if (dd > 0.f) hi = (uint32_t)(((unsigned long long)first_offset_reaching(dd, 1.f) << 8) - 1ull);
    if (dd < 0.f) lo = (uint32_t)((unsigned long long)first_offset_reaching(dd, 0.f) << 8);
    xlo[e] = lo;
    xhi[e] = hi;
  }
  for (long long e = tid; e < sine_elems; e += nt) {
    const SimDesc& s = d[owner(d, n, e, 2)];
    const long long q = e - s.sine_off;
    sine[e] = sine_entry_n1(s.Q, (int)(q / s.Np), (int)(q % s.Np));
  }
}

// ---------------------------------------------------------------- per-cell scan
__global__ void k_b_rows(const int32_t* __restrict__ hist, const SimDesc* __restrict__ d,
                         const int* __restrict__ cell_sim, const float* __restrict__ D, long long n_cells,
                         unsigned long long* __restrict__ T, unsigned char* __restrict__ reach) {
  const long long c = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= n_cells) return;
  const SimDesc& s = d[__ldg(cell_sim + c)];
  const long long i = c - s.cell_off;
  const int n_M = s.n_M;
  const int32_t* row = hist + s.hist_off + i * n_M;
  // the drift D[M] = fl32(M d1), d1 > 0, has the sign of M: a column right of
  // the centre drifts right, left of it left (a D that rounds to zero only
  // marks a neighbour that needs its kernel anyway, which changes no result)
  unsigned long long a = 0;
  unsigned bits = 0;
  if ((n_M & 3) == 0 && (reinterpret_cast<uintptr_t>(row) & 15) == 0) {
    const int4* row4 = reinterpret_cast<const int4*>(row);
    for (int q = lane; q < n_M / 4; q += 32) {
      const int4 n4 = __ldg(row4 + q);
      const int nv[4] = {n4.x, n4.y, n4.z, n4.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (nv[e]) {
          const int M = 4 * q + e - n_M / 2;
          a += (unsigned long long)(nv[e] < 0 ? -(long long)nv[e] : (long long)nv[e]);
          bits |= 1u | (M > 0 ? 2u : 0u) | (M < 0 ? 4u : 0u);
        }
      }
    }
  } else {
    for (int k = lane; k < n_M; k += 32) {
      const int nv = __ldg(row + k);
      if (nv) {
        const int M = k - n_M / 2;
        a += (unsigned long long)(nv < 0 ? -(long long)nv : (long long)nv);
        bits |= 1u | (M > 0 ? 2u : 0u) | (M < 0 ? 4u : 0u);
      }
    }
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, off);
    bits |= __shfl_down_sync(0xffffffffu, bits, off);
  }
  if (lane == 0) {
    T[c] = a;
    reach[c] = (unsigned char)bits;
  }
}

// kernel needed at cell c: occupied, or a neighbour of the same simulation
// drifts into it
__device__ __forceinline__ int b_needs(const unsigned char* __restrict__ reach, const SimDesc* __restrict__ d,
                                       const int* __restrict__ cell_sim, long long c) {
  const SimDesc& s = d[__ldg(cell_sim + c)];
  const long long i = c - s.cell_off;
  return (reach[c] & 1) || (i > 0 && (reach[c - 1] & 2)) || (i + 1 < s.n_x && (reach[c + 1] & 4));
}

__device__ __forceinline__ int b_items(unsigned long long t, int chunk) {
  return t ? (int)((t + 3 + chunk - 1) / chunk) : 0;
}

// block-wide exclusive scan of three counters (256 threads)
__device__ __forceinline__ void block_scan3(unsigned long long& a, unsigned long long& b, unsigned long long& c,
                                            unsigned long long* sh /*3 x 8*/, unsigned long long tot[3]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long ia = a, ib = b, ic = c;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned long long ua = __shfl_up_sync(0xffffffffu, ia, off);
    const unsigned long long ub = __shfl_up_sync(0xffffffffu, ib, off);
    const unsigned long long uc = __shfl_up_sync(0xffffffffu, ic, off);
    if (lane >= off) {
      ia += ua;
      ib += ub;
      ic += uc;
    }
  }
  if (lane == 31) {
    sh[wid] = ia;
    sh[8 + wid] = ib;
    sh[16 + wid] = ic;
  }
  __syncthreads();
  unsigned long long pa = 0, pb = 0, pc = 0, ta = 0, tb = 0, tc = 0;
  for (int w = 0; w < 8; ++w) {
    if (w < wid) {
      pa += sh[w];
      pb += sh[8 + w];
      pc += sh[16 + w];
    }
    ta += sh[w];
    tb += sh[8 + w];
    tc += sh[16 + w];
  }
  a = pa + ia - a;
  b = pb + ib - b;
  c = pc + ic - c;
  tot[0] = ta;
  tot[1] = tb;
  tot[2] = tc;
}

constexpr int kCellsPerThread = kScanCells / kScanThreads;

__global__ __launch_bounds__(kScanThreads) void k_b_scan1(const unsigned long long* __restrict__ T,
                                                          const unsigned char* __restrict__ reach,
                                                          const SimDesc* __restrict__ d,
                                                          const int* __restrict__ cell_sim, long long n_cells,
                                                          int chunk, unsigned long long* __restrict__ blk) {
  __shared__ unsigned long long sh[24];
  const long long c0 = (long long)blockIdx.x * kScanCells + threadIdx.x * kCellsPerThread;
  unsigned long long a = 0, b = 0, c = 0;
  for (int q = 0; q < kCellsPerThread; ++q) {
    const long long cc = c0 + q;
    if (cc >= n_cells) break;
    const unsigned long long t = T[cc];
    a += t;
    b += b_items(t, chunk);
    c += b_needs(reach, d, cell_sim, cc);
  }
  unsigned long long tot[3];
  block_scan3(a, b, c, sh, tot);
  if (threadIdx.x == 0) {
    blk[3 * blockIdx.x] = tot[0];
    blk[3 * blockIdx.x + 1] = tot[1];
    blk[3 * blockIdx.x + 2] = tot[2];
  }
}

// single block: exclusive scan of the block sums, totals to the header
__global__ __launch_bounds__(kScanThreads) void k_b_scan2(unsigned long long* __restrict__ blk, int n_blk,
                                                          long long max_items, DevHeader* hdr, int advance_step) {
  __shared__ unsigned long long sh[24];
  __shared__ unsigned long long carry[3];
  if (threadIdx.x == 0) carry[0] = carry[1] = carry[2] = 0;
  __syncthreads();
  for (int base = 0; base < n_blk; base += kScanThreads) {
    const int q = base + threadIdx.x;
    unsigned long long a = 0, b = 0, c = 0;
    if (q < n_blk) {
      a = blk[3 * q];
      b = blk[3 * q + 1];
      c = blk[3 * q + 2];
    }
    unsigned long long tot[3];
    block_scan3(a, b, c, sh, tot);
    if (q < n_blk) {
      blk[3 * q] = a + carry[0];
      blk[3 * q + 1] = b + carry[1];
      blk[3 * q + 2] = c + carry[2];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      carry[0] += tot[0];
      carry[1] += tot[1];
      carry[2] += tot[2];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int ok = (long long)carry[1] <= max_items;
    hdr->n_items = ok ? (int)carry[1] : 0;
    hdr->n_occ = (int)carry[2];
    hdr->population = 0;  // summed per simulation by k_b_simbase
    if (!ok) atomicOr(&hdr->flags, WMC_FLAG_CAPACITY);
    if (advance_step) hdr->step += 1u;
  }
}

__global__ __launch_bounds__(kScanThreads) void k_b_scan3(
    const unsigned long long* __restrict__ T, const unsigned char* __restrict__ reach, const SimDesc* __restrict__ d,
    const int* __restrict__ cell_sim, long long n_cells, int chunk, const unsigned long long* __restrict__ blk,
    unsigned long long* __restrict__ G, int2* __restrict__ items, int* __restrict__ occ, int* __restrict__ row_map,
    unsigned long long* __restrict__ thr_cell, DevHeader* hdr) {
  __shared__ unsigned long long sh[24];
  const long long c0 = (long long)blockIdx.x * kScanCells + threadIdx.x * kCellsPerThread;
  unsigned long long a = 0, b = 0, c = 0;
  for (int q = 0; q < kCellsPerThread; ++q) {
    const long long cc = c0 + q;
    if (cc >= n_cells) break;
    const unsigned long long t = T[cc];
    a += t;
    b += b_items(t, chunk);
    c += b_needs(reach, d, cell_sim, cc);
  }
  unsigned long long tot[3];
  block_scan3(a, b, c, sh, tot);
  a += blk[3 * blockIdx.x];
  b += blk[3 * blockIdx.x + 1];
  c += blk[3 * blockIdx.x + 2];
  const bool write_items = hdr->n_items > 0;
  for (int q = 0; q < kCellsPerThread; ++q) {
    const long long cc = c0 + q;
    if (cc >= n_cells) break;
    const unsigned long long t = T[cc];
    G[cc] = a;
    if (t > 0x7fffffffull) {  // a cell's ids must fit the 31-bit row-local offsets
      atomicOr(&hdr->flags, WMC_FLAG_CAPACITY);
      hdr->n_items = 0;
    }
    const int ni = b_items(t, chunk);
    if (write_items)
      for (int k = 0; k < ni; ++k) items[b + k] = make_int2((int)cc, k);
    if (b_needs(reach, d, cell_sim, cc)) {
      occ[c] = (int)cc;
      row_map[cc] = (int)c;
      ++c;
    } else {
      row_map[cc] = -1;
    }
    thr_cell[cc] = 0ull;
    a += t;
    b += ni;
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) G[n_cells] = blk[3 * blockIdx.x] + tot[0];
}

// per simulation: first id offset and population
__global__ void k_b_simbase(const SimDesc* __restrict__ d, int n, const unsigned long long* __restrict__ G,
                            unsigned long long* __restrict__ base, DevHeader* hdr) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const unsigned long long b0 = G[d[s].cell_off], b1 = G[d[s].cell_off + d[s].n_x];
  base[s] = b0;
  const unsigned long long P = b1 - b0;
  atomicAdd(&hdr->population, P);
  if (P >= (1ull << 32)) {  // ids of one simulation are 32-bit
    atomicOr(&hdr->flags, WMC_FLAG_CAPACITY);
    hdr->n_items = 0;
  }
}

// ---------------------------------------------------------------- kernel rows
// One warp per occupied cell of any simulation: FP32 contraction with the
// simulation's own window and sine matrix (read through L1), then the
// fixed-point CDF, gamma and event threshold of the row.
template <int C>
__global__ __launch_bounds__(kBatchRowWarps * 32) void k_b_kernel_rows(
    const float* __restrict__ V, const SimDesc* __restrict__ d, const int* __restrict__ cell_sim,
    const int* __restrict__ occ, const DevHeader* __restrict__ hdr, const float* __restrict__ sine, int H, int NM,
    float* __restrict__ VWh, long long* __restrict__ cdf, double* __restrict__ gamma,
    unsigned long long* __restrict__ gthr, unsigned long long* __restrict__ thr_cell, unsigned int* __restrict__ flags) {
  __shared__ float s_buf[kBatchRowWarps][2 * 32 * C];
  const int n_rows = hdr->n_occ;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* s_row = s_buf[wid];
  float* s_dv = s_buf[wid] + 32 * C;
  for (int row = blockIdx.x * kBatchRowWarps + wid; row < n_rows; row += gridDim.x * kBatchRowWarps) {
    const int cg = __ldg(occ + row);
    const SimDesc& s = d[__ldg(cell_sim + cg)];
    const int i = (int)(cg - s.cell_off), h = s.h, Q = s.Q, n_M = s.n_M;
    const float* Vs = V + s.cell_off;
    const float* B = sine + s.sine_off;
#pragma unroll
    for (int q = 0; q < C; ++q) {
      const int m = lane + 1 + 32 * q;
      s_dv[m - 1] = m <= h - 1 ? __fsub_rn(pot(Vs, s.n_x, s.bc, (long long)i + m), pot(Vs, s.n_x, s.bc, (long long)i - m))
                               : 0.f;
    }
    bool nz = false;  // a flat potential over the window gives an exactly zero row: skip the sums
#pragma unroll
    for (int q = 0; q < C; ++q) nz |= s_dv[lane + 32 * q] != 0.f;
    nz = __any_sync(0xffffffffu, nz);
    __syncwarp();
    float sacc[C], eacc[C];
#pragma unroll
    for (int cc = 0; cc < C; ++cc) sacc[cc] = eacc[cc] = 0.f;
    for (int m0 = 1; nz && m0 <= h - 1; m0 += 32) {
      float part[C];
#pragma unroll
      for (int cc = 0; cc < C; ++cc) part[cc] = 0.f;
      const int m1 = min(m0 + 32, h);
      for (int m = m0; m < m1; ++m) {
        const float dv = s_dv[m - 1];
        const float* brow = B + (size_t)(m - 1) * s.Np;
#pragma unroll
        for (int cc = 0; cc < C; ++cc) {
          const int r = lane + 32 * cc;
          if (r < h) part[cc] = fmaf(dv, __ldg(brow + r), part[cc]);
        }
      }
#pragma unroll
      for (int cc = 0; cc < C; ++cc) two_sum_acc(sacc[cc], eacc[cc], part[cc]);
    }
    float* out = VWh + (size_t)row * H;
#pragma unroll
    for (int cc = 0; cc < C; ++cc) {
      const int r = lane + 32 * cc;
      if (r < h) {
        const float v = __fmul_rn(s.c, __fadd_rn(sacc[cc], eacc[cc]));
        out[r] = v;
        s_row[r] = v;
      }
    }
    __syncwarp();
    const int r0 = ((-(n_M / 2)) % Q + Q) % Q;
    auto xres = [&](int rr) { return positive_part_smem(s_row, Q, rr); };
    double g;
    int sc;
    long long tot;
    warp_row_cdf(xres, Q, r0, n_M, s.log2_nM, lane, cdf + (size_t)row * NM, g, sc, tot, false);
    if (lane == 0) {
      gamma[row] = g;
      const unsigned long long thr = g > 0.0 ? event_threshold(g, s.dt, flags) : 0ull;
      gthr[row] = thr;
      thr_cell[cg] = thr;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------- step
struct BatchStepArgs {
  const int32_t* hist_in;
  int32_t* hist_out;
  const SimDesc* d;
  const int* cell_sim;
  const unsigned long long* G;
  const unsigned long long* sim_base;
  const int2* items;
  const int* row_map;
  const long long* cdf;
  const unsigned long long* thr_cell;
  const uint32_t* xlo;
  const uint32_t* xhi;
  DevHeader* hdr;
  int NM, per_thread;
};

// One warp per work item: an item is a run of 32 x per_thread ids of one row
// (quad-aligned to the global ids), so a sparse row costs one warp, not a
// block.  Each warp owns its slice of shared memory (row prefix and signed
// counts) and takes items from the global ticket without block-wide barriers;
// parents and children go to the output histogram with global atomics, one
// per run of ids in a bucket (lanes ending in the same bucket combine first),
// so a sparse item touches only the buckets it holds.
constexpr int kBStepWarps = 8;

__global__ __launch_bounds__(kBStepWarps * 32, 4) void k_b_step(BatchStepArgs a) {
  extern __shared__ int smem[];
  const int NM = a.NM;
  const int tid = threadIdx.x, lane = tid & 31;
  int* s_pre = smem + (size_t)(tid >> 5) * (2 * NM + 1);
  int* s_n = s_pre + (NM + 1);
  __shared__ unsigned long long s_red[5][kBStepWarps];
  const uint32_t t = a.hdr->step;
  const int n_items = a.hdr->n_items;
  const int PER = a.per_thread;
  const int chunk = 32 * PER;
  unsigned long long pairs = 0, absorbed = 0, dropped = 0;
  long long abs_signed = 0, drop_signed = 0;

  for (;;) {
    int item = 0;
    if (lane == 0) item = (int)atomicAdd(&a.hdr->item_ticket, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= n_items) break;
    const int2 it = __ldg(a.items + item);
    const long long cg = it.x;
    const int ch = it.y;
    const int sidx = __ldg(a.cell_sim + cg);
    const SimDesc& S = a.d[sidx];
    const int n_M = S.n_M, n_x = S.n_x;
    const int i = (int)(cg - S.cell_off);
    const uint32_t base = (uint32_t)(__ldg(a.G + cg) - __ldg(a.sim_base + sidx));
    const unsigned long long thr_m = i > 0 ? __ldg(a.thr_cell + cg - 1) : 0ull;
    const unsigned long long thr_0 = __ldg(a.thr_cell + cg);
    const unsigned long long thr_p = i + 1 < n_x ? __ldg(a.thr_cell + cg + 1) : 0ull;
    const uint32_t sim = S.sim, k0 = S.k0, k1 = S.k1;
    const int32_t* hrow = a.hist_in + S.hist_off;
    int32_t* hout = a.hist_out + S.hist_off + (size_t)(i - 1) * n_M;  // rows i-1, i, i+1 at hout + d n_M
    const uint32_t* xlo = a.xlo + S.tab_off;
    const uint32_t* xhi = a.xhi + S.tab_off;
    warp_row_prefix(hrow, i, n_M, s_n, s_pre, lane);
    __syncwarp();

    const uint32_t Ti = (uint32_t)s_pre[n_M];
    // the item is [item0, item1) of the quad-aligned id range of the cell; its
    // ids are spread over the 32 lanes in quad-aligned spans, so a sparse cell
    // keeps every lane busy
    const unsigned long long A = base & ~3u;
    const unsigned long long row_end = (unsigned long long)base + Ti;
    const unsigned long long item0 = A + (unsigned long long)ch * chunk;
    const unsigned long long item1 = item0 + chunk < row_end ? item0 + chunk : row_end;
    const unsigned long long len = item1 > item0 ? item1 - item0 : 0ull;
    const unsigned long long span = ((len + 127ull) / 128ull) * 4ull;
    const unsigned long long lo64 = item0 + (unsigned long long)lane * span;
    const unsigned long long g0_64 = lo64 > base ? lo64 : base;
    const unsigned long long g1_64 = lo64 + span < item1 ? lo64 + span : item1;
    const uint32_t g0 = g0_64 < g1_64 ? (uint32_t)g0_64 : 0u;
    const uint32_t g1 = g0_64 < g1_64 ? (uint32_t)g1_64 : 0u;
    const bool need_gen = (thr_m | thr_0 | thr_p) != 0ull;

    int k = 0, n_tot = 0, n_mov = 0, sgn = 1, dir = 0;
    if (g0 < g1) {
      k = bucket_of(s_pre, n_M, (int)(g0 - base));
      uint32_t end_g = base + (uint32_t)s_pre[k + 1];
      sgn = s_n[k] > 0 ? 1 : -1;
      uint32_t lo = __ldg(xlo + k), hi = __ldg(xhi + k);
      dir = drift_dir(lo, hi);
      unsigned long long thr_move = dir > 0 ? thr_p : (dir < 0 ? thr_m : 0ull);
      for (uint32_t q = g0 >> 2; q <= (g1 - 1u) >> 2; ++q) {
        const uint32_t qa = q << 2;
        const uint4 wr = philox4x32_10(make_uint4(q, t - 1u, kPurposeRepos, sim), k0, k1);
        uint4 wg = make_uint4(0u, 0u, 0u, 0u);
        if (need_gen) wg = philox4x32_10(make_uint4(q, t, kPurposeGen, sim), k0, k1);
        const uint32_t w4[4] = {wr.x, wr.y, wr.z, wr.w};
        const uint32_t u4[4] = {wg.x, wg.y, wg.z, wg.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t id = qa + (uint32_t)j;
          if (id < g0 || id >= g1) continue;
          if (id >= end_g) {
            const int stay = n_tot - n_mov;
            if (stay) atomicAdd(hout + (size_t)n_M + k, sgn * stay);
            if (n_mov) {
              if ((unsigned)(i + dir) < (unsigned)n_x) {
                atomicAdd(hout + (size_t)(dir + 1) * n_M + k, sgn * n_mov);
              } else {
                absorbed += n_mov;
                abs_signed += sgn * n_mov;
              }
            }
            n_tot = n_mov = 0;
            do { ++k; } while (base + (uint32_t)s_pre[k + 1] <= id);
            end_g = base + (uint32_t)s_pre[k + 1];
            sgn = s_n[k] > 0 ? 1 : -1;
            lo = __ldg(xlo + k);
            hi = __ldg(xhi + k);
            dir = drift_dir(lo, hi);
            thr_move = dir > 0 ? thr_p : (dir < 0 ? thr_m : 0ull);
          }
          const int mv = (w4[j] > hi) | (w4[j] < lo);
          n_mov += mv;
          ++n_tot;
          if (need_gen && (unsigned long long)u4[j] < (mv ? thr_move : thr_0)) {
            // pair: p' from the PICK draw of this id, children into row d
            const int dd = mv ? dir + 1 : 1;
            const int orow = __ldg(a.row_map + cg - 1 + dd);
            const uint4 wp = philox4x32_10(make_uint4(id, t, kPurposePick, sim), k0, k1);
            const unsigned long long U2 =
                ((unsigned long long)(wp.x >> 5) << 26) | (unsigned long long)(wp.y >> 6);
            const int kp = sample_cdf_row(a.cdf + (size_t)orow * NM, n_M, U2);
            ++pairs;
            const int Mp = kp - n_M / 2;
            const int kc2[2] = {k + Mp, k - Mp};
            const int sc2[2] = {sgn, -sgn};
#pragma unroll
            for (int qq = 0; qq < 2; ++qq) {
              int kc = kc2[qq];
              if (kc < 0 || kc >= n_M) {
                if (!S.wrap) {
                  ++dropped;
                  drop_signed += sc2[qq];
                  continue;
                }
                kc = ((kc % n_M) + n_M) % n_M;
              }
              atomicAdd(hout + (size_t)dd * n_M + kc, sc2[qq]);
            }
          }
        }
      }
    }
    const int key = n_tot ? k : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int stay = __reduce_add_sync(peers, n_tot - n_mov);
    const int mov = __reduce_add_sync(peers, n_mov);
    if (key >= 0 && lane == __ffs(peers) - 1) {
      if (stay) atomicAdd(hout + (size_t)n_M + k, sgn * stay);
      if (mov) {
        if ((unsigned)(i + dir) < (unsigned)n_x) {
          atomicAdd(hout + (size_t)(dir + 1) * n_M + k, sgn * mov);
        } else {
          absorbed += mov;
          abs_signed += sgn * mov;
        }
      }
    }
    __syncwarp();
  }
  const int wid = tid >> 5;
  unsigned long long vals[5] = {pairs, absorbed, (unsigned long long)abs_signed, dropped,
                                (unsigned long long)drop_signed};
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    unsigned long long v = vals[j];
#pragma unroll
    for (int off = 16; off; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) s_red[j][wid] = v;
  }
  __syncthreads();
  if (tid < 5) {
    unsigned long long v = 0;
    for (int w = 0; w < kBStepWarps; ++w) v += s_red[tid][w];
    if (v) {
      unsigned long long* dst[5] = {&a.hdr->pairs, &a.hdr->absorbed,
                                    reinterpret_cast<unsigned long long*>(&a.hdr->absorbed_signed), &a.hdr->dropped,
                                    reinterpret_cast<unsigned long long*>(&a.hdr->dropped_signed)};
      atomicAdd(dst[tid], v);
    }
  }
  if (blockIdx.x == 0 && tid == 0 && n_items > 0) atomicAdd(&a.hdr->particle_steps, a.hdr->population);
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&a.hdr->blocks_done, 1u) == gridDim.x - 1) {
      a.hdr->item_ticket = 0u;
      a.hdr->blocks_done = 0u;
      __threadfence();
    }
  }
}

__global__ void k_b_set_step(DevHeader* hdr, uint32_t step) { hdr->step = step; }

// ---------------------------------------------------------------- host driver
size_t b_step_smem(int NM) { return sizeof(int) * (size_t)kBStepWarps * (2 * NM + 1); }

int b_step_grid(int NM) {
  int per_sm = 0;
  const size_t sm = b_step_smem(NM);
  if (sm > 48 * 1024) raise_smem_limit(reinterpret_cast<const void*>(k_b_step), sm);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_b_step, kBStepWarps * 32, sm);
  if (per_sm < 1) per_sm = 1;
  return per_sm * num_sms();
}

cudaError_t b_one_step(const BatchLayout& L, const BatchView& v, int n, const float* V, const int32_t* in,
                       int32_t* out, int per_thread, int grid, cudaStream_t s) {
  const long long nc = L.n_cells;
  const int chunk = 32 * per_thread;  // ids per warp item
  k_b_rows<<<(unsigned)((nc * 32 + 255) / 256), 256, 0, s>>>(in, v.descs, v.cell_sim, v.D, nc, v.T, v.reach);
  k_b_scan1<<<L.n_blk, kScanThreads, 0, s>>>(v.T, v.reach, v.descs, v.cell_sim, nc, chunk, v.blk);
  k_b_scan2<<<1, kScanThreads, 0, s>>>(v.blk, L.n_blk, L.max_items, v.hdr, 1);
  k_b_scan3<<<L.n_blk, kScanThreads, 0, s>>>(v.T, v.reach, v.descs, v.cell_sim, nc, chunk, v.blk, v.G, v.items, v.occ,
                                             v.row_map, v.thr_cell, v.hdr);
  k_b_simbase<<<(n + 127) / 128, 128, 0, s>>>(v.descs, n, v.G, v.sim_base, v.hdr);
  const int rows_blocks = (int)((nc + kBatchRowWarps - 1) / kBatchRowWarps);
  const int rb = rows_blocks < 8 * num_sms() ? rows_blocks : 8 * num_sms();
  if (L.H <= 32)
    k_b_kernel_rows<1><<<rb, kBatchRowWarps * 32, 0, s>>>(V, v.descs, v.cell_sim, v.occ, v.hdr, v.sine, L.H, L.NM,
                                                          v.VWh, v.cdf, v.gamma, v.gthr, v.thr_cell, &v.hdr->flags);
  else if (L.H <= 64)
    k_b_kernel_rows<2><<<rb, kBatchRowWarps * 32, 0, s>>>(V, v.descs, v.cell_sim, v.occ, v.hdr, v.sine, L.H, L.NM,
                                                          v.VWh, v.cdf, v.gamma, v.gthr, v.thr_cell, &v.hdr->flags);
  else
    k_b_kernel_rows<4><<<rb, kBatchRowWarps * 32, 0, s>>>(V, v.descs, v.cell_sim, v.occ, v.hdr, v.sine, L.H, L.NM,
                                                          v.VWh, v.cdf, v.gamma, v.gthr, v.thr_cell, &v.hdr->flags);
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int32_t) * (size_t)L.hist_elems, s);
  if (e != cudaSuccess) return e;
  BatchStepArgs a;
  a.hist_in = in;
  a.hist_out = out;
  a.d = v.descs;
  a.cell_sim = v.cell_sim;
  a.G = v.G;
  a.sim_base = v.sim_base;
  a.items = v.items;
  a.row_map = v.row_map;
  a.cdf = v.cdf;
  a.thr_cell = v.thr_cell;
  a.xlo = v.xlo;
  a.xhi = v.xhi;
  a.hdr = v.hdr;
  a.NM = L.NM;
  a.per_thread = per_thread;
  k_b_step<<<grid, kBStepWarps * 32, b_step_smem(L.NM), s>>>(a);
  return cudaGetLastError();
}

struct BatchGraph {
  std::mutex mu;
  bool valid = false;
  std::vector<wmc_params> ps;
  const void *V, *a, *b, *ws;
  int per;
  cudaStream_t stream;
  int device;
  cudaGraphExec_t exec = nullptr;
};
BatchGraph g_bgraph;

bool valid_per(int per) { return per == 4 || per == 8 || per == 16 || per == 32 || per == 64 || per == 128 || per == 256; }

}  // namespace
}  // namespace wmc

using namespace wmc;

extern "C" {

size_t wmc_batch_workspace_size(const wmc_params* ps, int32_t n_sims) {
  if (!batch_ok(ps, n_sims)) return 0;
  return batch_layout(ps, n_sims).total;
}

wmc_status wmc_batch_layout(const wmc_params* ps, int32_t n_sims, int64_t* cell_off, int64_t* hist_off) {
  if (!batch_ok(ps, n_sims) || !cell_off || !hist_off) return WMC_ERR_ARG;
  long long c = 0, h = 0;
  for (int s = 0; s < n_sims; ++s) {
    cell_off[s] = c;
    hist_off[s] = h;
    c += ps[s].n_x;
    h += (long long)ps[s].n_x * ps[s].n_M;
  }
  cell_off[n_sims] = c;
  hist_off[n_sims] = h;
  return WMC_OK;
}

wmc_status wmc_batch_init(const wmc_params* ps, int32_t n_sims, void* ws, size_t ws_bytes, wmc_stream_t stream) {
  if (!batch_ok(ps, n_sims) || !ws || ((uintptr_t)ws & 255)) return WMC_ERR_ARG;
  const BatchLayout L = batch_layout(ps, n_sims);
  if (ws_bytes < L.total) return WMC_ERR_ARG;
  std::vector<SimDesc> d(n_sims);
  long long c = 0, h = 0, tb = 0, sn = 0;
  for (int s = 0; s < n_sims; ++s) {
    const wmc_params& p = ps[s];
    SimDesc& x = d[s];
    memset(&x, 0, sizeof(x));
    x.n_x = p.n_x;
    x.Q = p.Q;
    x.n_M = p.n_M;
    x.bc = p.bc_potential;
    x.wrap = p.child_wrap;
    x.h = p.Q / 2;
    x.log2_nM = ceil_log2_host(p.n_M);
    x.Kp = ((x.h - 1 + 31) / 32) * 32 > 0 ? ((x.h - 1 + 31) / 32) * 32 : 32;
    x.Np = ((x.h + 63) / 64) * 64;
    x.sim = p.sim;
    x.k0 = (uint32_t)(p.seed & 0xffffffffu);
    x.k1 = (uint32_t)(p.seed >> 32);
    x.c = (float)(-2.0 / (kHbarEVs * (double)p.Q));
    x.dt = p.dt_s;
    x.d1 = ((kHbarJs * kPi) * p.dt_s) / ((p.mass_kg * (double)p.Q) * (p.dx_m * p.dx_m));
    x.cell_off = c;
    x.hist_off = h;
    x.tab_off = tb;
    x.sine_off = sn;
    c += p.n_x;
    h += (long long)p.n_x * p.n_M;
    tb += p.n_M;
    sn += (long long)x.Kp * x.Np;
  }
  const BatchView v = batch_view(L, ws);
  cudaStream_t s = (cudaStream_t)stream;
  // set-up copy of the descriptors (synchronous: the host vector is temporary)
  if (cudaMemcpyAsync(v.descs, d.data(), sizeof(SimDesc) * n_sims, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return WMC_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return WMC_ERR_CUDA;
  k_b_init<<<512, 256, 0, s>>>(v.descs, n_sims, L.n_cells, L.tab_elems, L.sine_elems, v.cell_sim, v.D, v.xlo, v.xhi,
                               v.sine, v.hdr);
  (void)b_step_grid(L.NM);
  return cudaGetLastError() == cudaSuccess ? WMC_OK : WMC_ERR_CUDA;
}

wmc_status wmc_batch_run(const wmc_params* ps, int32_t n_sims, const float* V, int32_t* hist_a, int32_t* hist_b,
                         uint32_t t_first, int32_t n_steps, int32_t per_thread, int32_t use_graph, void* ws,
                         wmc_stream_t stream) {
  NvtxRange nvtx("wmc_batch_run");
  if (!batch_ok(ps, n_sims) || !V || !hist_a || !hist_b || hist_a == hist_b || !ws || n_steps < 0 || t_first == 0)
    return WMC_ERR_ARG;
  if (per_thread == 0) per_thread = 16;
  if (!valid_per(per_thread)) return WMC_ERR_ARG;
  if (n_steps == 0) return WMC_OK;
  const BatchLayout L = batch_layout(ps, n_sims);
  const BatchView v = batch_view(L, ws);
  cudaStream_t s = (cudaStream_t)stream;
  const int grid = b_step_grid(L.NM);
  k_b_set_step<<<1, 1, 0, s>>>(v.hdr, t_first - 1u);
  if (cudaGetLastError() != cudaSuccess) return WMC_ERR_CUDA;
  const int pairs = n_steps / 2;
  if (use_graph && s != nullptr && pairs > 0) {
    std::lock_guard<std::mutex> lock(g_bgraph.mu);
    int dev = 0;
    cudaGetDevice(&dev);
    bool hit = g_bgraph.valid && (int)g_bgraph.ps.size() == n_sims && g_bgraph.V == V && g_bgraph.a == hist_a &&
               g_bgraph.b == hist_b && g_bgraph.ws == ws && g_bgraph.per == per_thread && g_bgraph.stream == s &&
               g_bgraph.device == dev;
    if (hit) hit = memcmp(g_bgraph.ps.data(), ps, sizeof(wmc_params) * n_sims) == 0;
    if (!hit) {
      if (g_bgraph.exec) {
        cudaGraphExecDestroy(g_bgraph.exec);
        g_bgraph.exec = nullptr;
      }
      g_bgraph.valid = false;
      cudaGraph_t graph = nullptr;
      if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return WMC_ERR_CUDA;
      cudaError_t e = b_one_step(L, v, n_sims, V, hist_a, hist_b, per_thread, grid, s);
      if (e == cudaSuccess) e = b_one_step(L, v, n_sims, V, hist_b, hist_a, per_thread, grid, s);
      const cudaError_t e2 = cudaStreamEndCapture(s, &graph);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return WMC_ERR_CUDA;
      }
      e = cudaGraphInstantiate(&g_bgraph.exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return WMC_ERR_CUDA;
      g_bgraph.valid = true;
      g_bgraph.ps.assign(ps, ps + n_sims);
      g_bgraph.V = V;
      g_bgraph.a = hist_a;
      g_bgraph.b = hist_b;
      g_bgraph.ws = ws;
      g_bgraph.per = per_thread;
      g_bgraph.stream = s;
      g_bgraph.device = dev;
    }
    for (int q = 0; q < pairs; ++q)
      if (cudaGraphLaunch(g_bgraph.exec, s) != cudaSuccess) return WMC_ERR_CUDA;
  } else {
    for (int q = 0; q < pairs; ++q) {
      if (b_one_step(L, v, n_sims, V, hist_a, hist_b, per_thread, grid, s) != cudaSuccess) return WMC_ERR_CUDA;
      if (b_one_step(L, v, n_sims, V, hist_b, hist_a, per_thread, grid, s) != cudaSuccess) return WMC_ERR_CUDA;
    }
  }
  if (n_steps & 1) {
    if (b_one_step(L, v, n_sims, V, hist_a, hist_b, per_thread, grid, s) != cudaSuccess) return WMC_ERR_CUDA;
    if (cudaMemcpyAsync(hist_a, hist_b, sizeof(int32_t) * (size_t)L.hist_elems, cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
      return WMC_ERR_CUDA;
  }
  return WMC_OK;
}

wmc_status wmc_batch_autotune(const wmc_params* ps, int32_t n_sims, const float* V, int32_t* hist, int32_t* scratch,
                              uint32_t t, void* ws, int32_t* best_per_thread, wmc_stream_t stream) {
  if (!batch_ok(ps, n_sims) || !V || !hist || !scratch || hist == scratch || !ws || !best_per_thread || t == 0)
    return WMC_ERR_ARG;
  const BatchLayout L = batch_layout(ps, n_sims);
  const BatchView v = batch_view(L, ws);
  cudaStream_t s = (cudaStream_t)stream;
  const int grid = b_step_grid(L.NM);
  const int cands[5] = {16, 32, 64, 128, 256};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return WMC_ERR_CUDA;
  float best = 1e30f;
  int best_per = 16;
  for (int r = 0; r < 2; ++r) {  // second round measures warm
    for (int q = 0; q < 5; ++q) {
      k_b_set_step<<<1, 1, 0, s>>>(v.hdr, t - 1u);
      cudaEventRecord(e0, s);
      if (b_one_step(L, v, n_sims, V, hist, scratch, cands[q], grid, s) != cudaSuccess) return WMC_ERR_CUDA;
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) return WMC_ERR_CUDA;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r == 1 && ms < best) {
        best = ms;
        best_per = cands[q];
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *best_per_thread = best_per;
  return WMC_OK;
}

wmc_status wmc_batch_get_counters(const wmc_params* ps, int32_t n_sims, const void* ws, wmc_counters* out,
                                  wmc_stream_t stream) {
  if (!batch_ok(ps, n_sims) || !ws || !out) return WMC_ERR_ARG;
  const BatchLayout L = batch_layout(ps, n_sims);
  DevHeader h;
  const char* b = static_cast<const char*>(ws);
  cudaError_t e = cudaMemcpyAsync(&h, b + L.header, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
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
  return h.magic == kMagic ? WMC_OK : WMC_ERR_ARG;
}

}  // extern "C"
