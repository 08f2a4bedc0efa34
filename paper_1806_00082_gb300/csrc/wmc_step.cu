// One step of the postulate (Sec. 2.1) over the survivors of a net histogram:
// free drift, absorption, pair creation with probability gamma dt and momentum
// p' ~ V_W^+ / gamma, and the signed histogram of parents and children (whose
// summation is the annihilation of rule 2).
//
// The survivors are never stored: after annihilation every particle of bucket
// (i, M) carries the same cell, momentum and sign, and its offset is a Philox
// draw of its id, so the histogram and the id prefix describe the ensemble
// exactly.  A block takes work items (up to kChunk ids of one cell, aligned
// so that each Philox call serves four consecutive ids of one thread) in a
// fixed round-robin order; while its seven worker warps step the particles of
// one item, warp 0 loads the next item's descriptor and row prefix into the
// other of two shared buffers, so that latency is off the critical path.  The
// block privatises the three histogram rows its particles can land in (i-1, i,
// i+1) in shared memory and flushes them with one global atomic per non-zero
// bucket.  A particle moves iff its offset word passes the integer threshold
// of its momentum column, so a quad of ids inside one bucket costs one Philox
// call and a handful of compares.
#include "wmc_device.cuh"

namespace wmc {

struct StepArgs {
  const int32_t* hist_in;
  int32_t* hist_out;
  const unsigned long long* R;
  const int2* items;
  long long max_items;  // capacity of items
  const int* row_map;
  const long long* cdf;  // [rows][n_M] fixed-point CDF
  const unsigned long long* thr_cell;
  const uint32_t* xlo;
  const uint32_t* xhi;
  DevHeader* hdr;
  int n_x, n_M, Q, child_wrap;
  uint32_t sim, k0, k1, t;
  int t_from_device;
  int rows_by_cell;  // read from the header at kernel start
};

// Loads the signed counts of cell i into s_n and their exclusive prefix of
// |n| into s_pre[0..n_M] (s_pre[n_M] = survivors of the cell), block-wide.
__device__ __forceinline__ void load_row_prefix(const int32_t* __restrict__ hist, int i, int n_M, int* s_n,
                                                int* s_pre, int* s_wsum) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int E = (n_M + kStepThreads - 1) / kStepThreads;
  const int k0 = min(tid * E, n_M), k1 = min(k0 + E, n_M);
  const int32_t* row = hist + (size_t)i * n_M;
  int local = 0;
  for (int k = k0; k < k1; ++k) {
    const int n = row[k];
    s_n[k] = n;
    local += n < 0 ? -n : n;
  }
  int incl = local;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += u;
  }
  if (lane == 31) s_wsum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int w = lane < kStepThreads / 32 ? s_wsum[lane] : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += u;
    }
    if (lane < kStepThreads / 32) s_wsum[lane] = w;
  }
  __syncthreads();
  int excl = (wid ? s_wsum[wid - 1] : 0) + incl - local;
  for (int k = k0; k < k1; ++k) {
    s_pre[k] = excl;
    const int n = s_n[k];
    excl += n < 0 ? -n : n;
  }
  if (tid == kStepThreads - 1) s_pre[n_M] = s_wsum[kStepThreads / 32 - 1];
}

__device__ __forceinline__ int sample_momentum(const StepArgs& a, int orow, unsigned long long U2) {
  return sample_cdf_row(a.cdf + (size_t)orow * a.n_M, a.n_M, U2);
}

// A pair created by particle id (column k, sign sgn) that lands in cell c = i - 1 + d:
// p' from the PICK draw, children into the block's private row d.
__device__ __forceinline__ void create_pair(const StepArgs& a, uint32_t id, uint32_t t, int i, int d, int k,
                                            int sgn, int* s_acc, unsigned long long& pairs,
                                            unsigned long long& dropped, long long& drop_signed) {
  const int n_M = a.n_M;
  const int orow = a.rows_by_cell ? i - 1 + d : __ldg(a.row_map + i - 1 + d);
  const uint4 wp = philox4x32_10(make_uint4(id, t, kPurposePick, a.sim), a.k0, a.k1);
  const unsigned long long U2 = ((unsigned long long)(wp.x >> 5) << 26) | (unsigned long long)(wp.y >> 6);
  const int kp = sample_momentum(a, orow, U2);
  ++pairs;
  const int Mp = kp - n_M / 2;
  const int kc2[2] = {k + Mp, k - Mp};
  const int sc2[2] = {sgn, -sgn};
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    int kc = kc2[q];
    if (kc < 0 || kc >= n_M) {
      if (!a.child_wrap) {
        ++dropped;
        drop_signed += sc2[q];
        continue;
      }
      kc = ((kc % n_M) + n_M) % n_M;
    }
    atomicAdd(&s_acc[d * n_M + kc], sc2[q]);
  }
}

// Descriptor of a work item, prepared by warp 0 one item ahead.
struct ItemMeta {
  unsigned long long thr_m, thr_0, thr_p;  // event thresholds of cells i-1, i, i+1
  uint32_t base;                           // first id of cell i
  int item, i, ch;
};

__global__ __launch_bounds__(kStepThreads, 4) void k_step(StepArgs a) {
  extern __shared__ int smem[];
  a.rows_by_cell = (int)a.hdr->rows_by_cell;  // how the kernel stage laid out its CDF rows
  const int n_M = a.n_M;
  int* s_pre2 = smem;                    // 2 x (n_M + 1): prefix buffers
  int* s_n2 = s_pre2 + 2 * (n_M + 1);    // 2 x n_M: signed count buffers
  int* s_acc = s_n2 + 2 * n_M;           // 3 n_M: rows i-1, i, i+1
  uint32_t* s_lo = reinterpret_cast<uint32_t*>(s_acc + 3 * n_M);  // n_M
  uint32_t* s_hi = s_lo + n_M;                                     // n_M
  __shared__ ItemMeta s_meta[2];
  __shared__ unsigned long long s_red[5][kStepThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t t = a.t_from_device ? a.hdr->step : a.t;
  const int n_items = a.hdr->n_items;
  for (int k = tid; k < n_M; k += kStepThreads) {
    s_lo[k] = a.xlo[k];
    s_hi[k] = a.xhi[k];
  }
  for (int q = tid; q < 3 * n_M; q += kStepThreads) s_acc[q] = 0;

  // by warp 0: descriptor and row prefix of `item` into buffer `buf`
  auto prepare = [&](int item, int buf) {
    ItemMeta m;
    m.item = item;
    m.i = m.ch = 0;
    m.base = 0u;
    m.thr_m = m.thr_0 = m.thr_p = 0ull;
    // the descriptor load goes out before the item count is known (any index
    // below the capacity is readable; the count decides whether it is used)
    int2 it = make_int2(0, 0);
    if (item < a.max_items) it = __ldg(a.items + item);
    if (item < n_items) {
      m.i = it.x;
      m.ch = it.y;
      m.base = (uint32_t)__ldg(a.R + m.i);
      m.thr_m = m.i > 0 ? __ldg(a.thr_cell + m.i - 1) : 0ull;
      m.thr_0 = __ldg(a.thr_cell + m.i);
      m.thr_p = m.i + 1 < a.n_x ? __ldg(a.thr_cell + m.i + 1) : 0ull;
      warp_row_prefix(a.hist_in, m.i, n_M, s_n2 + buf * n_M, s_pre2 + buf * (n_M + 1), lane);
    }
    if (lane == 0) s_meta[buf] = m;
  };
  if (wid == 0) prepare(blockIdx.x, 0);

  unsigned long long pairs = 0, absorbed = 0, dropped = 0;
  long long abs_signed = 0, drop_signed = 0;

  for (int round = 0;; ++round) {
    __syncthreads();  // this item's buffer is ready; the previous item is flushed
    const int buf = round & 1;
    const ItemMeta m = s_meta[buf];
    if (m.item >= n_items) break;
    if (wid == 0) {
      prepare(m.item + (int)gridDim.x, buf ^ 1);
    } else {
      const int* s_pre = s_pre2 + buf * (n_M + 1);
      const int* s_n = s_n2 + buf * n_M;
      const int i = m.i, ch = m.ch;
      const uint32_t base = m.base;
      const unsigned long long thr_m = m.thr_m, thr_0 = m.thr_0, thr_p = m.thr_p;
      const int w = tid - 32;  // worker index
      const uint32_t Ti = (uint32_t)s_pre[n_M];
      // the item is [item0, item1) of the quad-aligned id range of the cell; its
      // ids are spread over all workers in quad-aligned spans (a cell's last,
      // partial item then keeps every worker busy too)
      const unsigned long long A = base & ~3u;
      const unsigned long long row_end = (unsigned long long)base + Ti;
      const unsigned long long item0 = A + (unsigned long long)ch * kChunk;
      const unsigned long long item1 = item0 + kChunk < row_end ? item0 + kChunk : row_end;
      const unsigned long long len = item1 > item0 ? item1 - item0 : 0ull;
      const unsigned long long span = ((len + 4ull * kStepWorkers - 1) / (4ull * kStepWorkers)) * 4ull;
      const unsigned long long lo64 = item0 + (unsigned long long)w * span;
      const unsigned long long g0_64 = lo64 > base ? lo64 : base;
      const unsigned long long g1_64 = lo64 + span < item1 ? lo64 + span : item1;
      // ids stay below 2^32 (the plan guarantees it); compare in 64 bits first
      const uint32_t g0 = g0_64 < g1_64 ? (uint32_t)g0_64 : 0u;
      const uint32_t g1 = g0_64 < g1_64 ? (uint32_t)g1_64 : 0u;
      const bool need_gen = (thr_m | thr_0 | thr_p) != 0ull;

      int k = 0, n_tot = 0, n_mov = 0, sgn = 1, dir = 0;
      if (g0 < g1) {
        k = bucket_of(s_pre, n_M, (int)(g0 - base));
        uint32_t end_g = base + (uint32_t)s_pre[k + 1];
        sgn = s_n[k] > 0 ? 1 : -1;
        uint32_t lo = s_lo[k], hi = s_hi[k];
        dir = drift_dir(lo, hi);
        unsigned long long thr_move = dir > 0 ? thr_p : (dir < 0 ? thr_m : 0ull);
        for (uint32_t q = g0 >> 2; q <= (g1 - 1u) >> 2; ++q) {
          const uint32_t qa = q << 2;
          const uint4 wr = philox4x32_10(make_uint4(q, t - 1u, kPurposeRepos, a.sim), a.k0, a.k1);
          uint4 wg = make_uint4(0u, 0u, 0u, 0u);
          if (need_gen) wg = philox4x32_10(make_uint4(q, t, kPurposeGen, a.sim), a.k0, a.k1);
          if (qa >= g0 && qa + 3u < g1 && qa + 3u < end_g) {
            // four consecutive ids of bucket k
            const int m0 = (wr.x > hi) | (wr.x < lo), m1 = (wr.y > hi) | (wr.y < lo);
            const int m2 = (wr.z > hi) | (wr.z < lo), m3 = (wr.w > hi) | (wr.w < lo);
            n_mov += m0 + m1 + m2 + m3;
            n_tot += 4;
            if (need_gen) {
              const int mv[4] = {m0, m1, m2, m3};
              const uint32_t u[4] = {wg.x, wg.y, wg.z, wg.w};
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                if ((unsigned long long)u[j] < (mv[j] ? thr_move : thr_0))
                  create_pair(a, qa + (uint32_t)j, t, i, mv[j] ? dir + 1 : 1, k, sgn, s_acc, pairs, dropped,
                              drop_signed);
              }
            }
            continue;
          }
          const uint32_t w4[4] = {wr.x, wr.y, wr.z, wr.w};
          const uint32_t u4[4] = {wg.x, wg.y, wg.z, wg.w};
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const uint32_t id = qa + (uint32_t)j;
            if (id < g0 || id >= g1) continue;
            if (id >= end_g) {  // next non-empty bucket
              const int stay = n_tot - n_mov;
              if (stay) atomicAdd(&s_acc[n_M + k], sgn * stay);
              if (n_mov) {
                if ((unsigned)(i + dir) < (unsigned)a.n_x) {
                  atomicAdd(&s_acc[(dir + 1) * n_M + k], sgn * n_mov);
                } else {
                  absorbed += n_mov;
                  abs_signed += sgn * n_mov;
                }
              }
              n_tot = n_mov = 0;
              do { ++k; } while (base + (uint32_t)s_pre[k + 1] <= id);
              end_g = base + (uint32_t)s_pre[k + 1];
              sgn = s_n[k] > 0 ? 1 : -1;
              lo = s_lo[k];
              hi = s_hi[k];
              dir = drift_dir(lo, hi);
              thr_move = dir > 0 ? thr_p : (dir < 0 ? thr_m : 0ull);
            }
            const int mv = (w4[j] > hi) | (w4[j] < lo);
            n_mov += mv;
            ++n_tot;
            if (need_gen && (unsigned long long)u4[j] < (mv ? thr_move : thr_0))
              create_pair(a, id, t, i, mv ? dir + 1 : 1, k, sgn, s_acc, pairs, dropped, drop_signed);
          }
        }
      }
      // last bucket of each thread: lanes holding the same bucket combine first
      const int key = n_tot ? k : -1;
      const unsigned peers = __match_any_sync(0xffffffffu, key);
      const int stay = __reduce_add_sync(peers, n_tot - n_mov);
      const int mov = __reduce_add_sync(peers, n_mov);
      if (key >= 0 && lane == __ffs(peers) - 1) {
        if (stay) atomicAdd(&s_acc[n_M + k], sgn * stay);
        if (mov) {
          if ((unsigned)(i + dir) < (unsigned)a.n_x) {
            atomicAdd(&s_acc[(dir + 1) * n_M + k], sgn * mov);
          } else {
            absorbed += mov;
            abs_signed += sgn * mov;
          }
        }
      }
    }
    __syncthreads();
    // flush the private rows (and clear them for the next item)
    for (int q = tid; q < 3 * n_M; q += kStepThreads) {
      const int v = s_acc[q];
      if (v) {
        s_acc[q] = 0;
        const int d = q / n_M, kc = q - d * n_M;
        atomicAdd(a.hist_out + (size_t)(m.i - 1 + d) * n_M + kc, v);
      }
    }
  }

  // block totals of the counters, one atomic each
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
    for (int w = 0; w < kStepThreads / 32; ++w) v += s_red[tid][w];
    if (v) {
      unsigned long long* dst[5] = {&a.hdr->pairs, &a.hdr->absorbed,
                                    reinterpret_cast<unsigned long long*>(&a.hdr->absorbed_signed), &a.hdr->dropped,
                                    reinterpret_cast<unsigned long long*>(&a.hdr->dropped_signed)};
      atomicAdd(dst[tid], v);
    }
  }
  if (blockIdx.x == 0 && tid == 0 && n_items > 0) atomicAdd(&a.hdr->particle_steps, a.hdr->population);
}

static size_t step_smem(int n_M) {
  return sizeof(int) * (size_t)(2 * (n_M + 1) + 2 * n_M + 3 * n_M) + 2 * sizeof(uint32_t) * n_M;
}

int step_grid(int n_M) {
  static int cached_nM[8] = {0};
  static int cached_grid[8] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  const int slot = dev & 7;
  if (cached_nM[slot] == n_M && cached_grid[slot] > 0) return cached_grid[slot];
  int per_sm = 0;
  const size_t sm = step_smem(n_M);
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step, kStepThreads, sm);
  if (per_sm < 1) per_sm = 1;
  int g = per_sm * num_sms();
  if (g > kMaxStepBlocks) g = kMaxStepBlocks;
  cached_nM[slot] = n_M;
  cached_grid[slot] = g;
  return g;
}

void prepare_step(const wmc_params& p) { (void)step_grid(p.n_M); }

cudaError_t launch_step(const wmc_params& p, const View& v, const int32_t* hist_in, uint32_t t, int t_from_device,
                        int32_t* hist_out, cudaStream_t s) {
  StepArgs a;
  a.hist_in = hist_in;
  a.hist_out = hist_out;
  a.R = v.R;
  a.items = v.items;
  a.max_items = layout(p).max_items;
  a.row_map = v.row_map;
  a.cdf = v.cdf;
  a.thr_cell = v.thr_cell;
  a.xlo = v.xlo;
  a.xhi = v.xhi;
  a.hdr = v.hdr;
  a.n_x = p.n_x;
  a.n_M = p.n_M;
  a.Q = p.Q;
  a.child_wrap = p.child_wrap;
  a.sim = p.sim;
  a.k0 = (uint32_t)(p.seed & 0xffffffffu);
  a.k1 = (uint32_t)(p.seed >> 32);
  a.t = t;
  a.t_from_device = t_from_device;
  a.rows_by_cell = 0;
  const int grid = step_grid(p.n_M);
  cudaError_t e = step_timing_record(s, false);
  if (e != cudaSuccess) return e;
  k_step<<<grid, kStepThreads, step_smem(p.n_M), s>>>(a);
  e = cudaGetLastError();
  return e == cudaSuccess ? step_timing_record(s, true) : e;
}

// ---------------------------------------------------------------- explicit survivors
__global__ __launch_bounds__(kStepThreads) void k_materialize(const int32_t* __restrict__ hist,
                                                              const unsigned long long* __restrict__ R,
                                                              const int* __restrict__ IP, DevHeader* hdr, int n_x,
                                                              int n_M, uint32_t sim, uint32_t k0, uint32_t k1,
                                                              uint32_t t, int32_t* __restrict__ cell,
                                                              float* __restrict__ f, int16_t* __restrict__ M,
                                                              int8_t* __restrict__ sign, long long capacity) {
  extern __shared__ int smem[];
  int* s_pre = smem;
  int* s_n = s_pre + (n_M + 1);
  __shared__ int s_wsum[kStepThreads / 32];
  __shared__ int s_row;
  const int tid = threadIdx.x;
  if ((long long)hdr->population > capacity) {
    if (blockIdx.x == 0 && tid == 0) atomicOr(&hdr->flags, WMC_FLAG_CAPACITY);
    return;
  }
  const int n_items = hdr->n_items;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    __syncthreads();
    if (tid == 0) {
      int lo = 0, hi = n_x;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(IP + mid) <= item) lo = mid; else hi = mid;
      }
      s_row = lo;
    }
    __syncthreads();
    const int i = s_row;
    const int chunk = item - __ldg(IP + i);
    load_row_prefix(hist, i, n_M, s_n, s_pre, s_wsum);
    __syncthreads();
    const int Ti = s_pre[n_M];
    const uint32_t base = (uint32_t)__ldg(R + i);
    const int lo = chunk * kChunk + tid * kPerThread;  // ids [chunk kChunk, (chunk + 1) kChunk) of the row
    const int hi = tid < kStepWorkers ? min(lo + kPerThread, Ti) : lo;
    if (lo < hi) {
      int k = bucket_of(s_pre, n_M, lo);
      for (int lid = lo; lid < hi; ++lid) {
        while (s_pre[k + 1] <= lid) ++k;
        const uint32_t id = base + (uint32_t)lid;
        const uint4 w = philox4x32_10(make_uint4(id >> 2, t, kPurposeRepos, sim), k0, k1);
        const uint32_t wj = (id & 3u) == 0u ? w.x : ((id & 3u) == 1u ? w.y : ((id & 3u) == 2u ? w.z : w.w));
        cell[id] = i;
        f[id] = (float)(wj >> 8) * 0x1p-24f;
        M[id] = (int16_t)(k - n_M / 2);
        sign[id] = (int8_t)(s_n[k] > 0 ? 1 : -1);
      }
    }
  }
}

cudaError_t launch_materialize(const wmc_params& p, const View& v, const int32_t* hist, uint32_t t, int32_t* cell,
                               float* f, int16_t* M, int8_t* sign, long long capacity, cudaStream_t s) {
  const size_t sm = sizeof(int) * (size_t)(2 * p.n_M + 1);
  k_materialize<<<2 * num_sms(), kStepThreads, sm, s>>>(hist, v.R, v.IP, v.hdr, p.n_x, p.n_M, p.sim,
                                                        (uint32_t)(p.seed & 0xffffffffu), (uint32_t)(p.seed >> 32),
                                                        t, cell, f, M, sign, capacity);
  return cudaGetLastError();
}

}  // namespace wmc
