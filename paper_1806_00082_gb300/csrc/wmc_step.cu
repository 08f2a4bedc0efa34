// One step of the postulate (Sec. 2.1) over the survivors of a net histogram:
// free drift, absorption, pair creation with probability gamma dt and momentum
// p' ~ V_W^+ / gamma, and the signed histogram of parents and children (whose
// summation is the annihilation of rule 2).
//
// The survivors are never stored: after annihilation every particle of bucket
// (i, M) carries the same cell, momentum and sign, and its offset is a Philox
// draw of its id, so the histogram and the id prefix describe the ensemble
// exactly.  Two kernels:
//   k_step   -- each warp takes work items (at most kChunk ids of one cell)
//               from a ticket counter, stages the cell's row prefix in its own
//               shared memory (no block barriers), and gives each lane a
//               quad-aligned run of ids: one Philox call per four ids for the
//               offsets (REPOS, step t - 1) and one for the pair-creation words
//               (GEN, step t) under a shared key schedule; a particle moves iff
//               its offset word passes the integer threshold of its momentum
//               column.  Parents are counted per bucket and added to the next
//               histogram with one reduction per bucket run; pair events are
//               queued in shared memory and appended to a global queue;
//   k_pairs  -- one thread per queued event: the PICK draw, p' from the coarse
//               CDF of the cell's kernel row, and the two children.
// Events beyond the queue's capacity are completed inside k_step (same
// arithmetic), so any rate is handled.
#include "wmc_device.cuh"

namespace wmc {

constexpr int kPairQ = 256;  // per-warp event queue (one quad iteration adds at most 128)
// a queue entry packs the id's offset in its item (13 bits), the column (12),
// the event cell relative to i - 1 (2) and the sign (1)
static_assert(kChunk <= 8192, "item offsets take 13 bits of a queue entry");

struct StepArgs {
  const int32_t* hist_in;
  int32_t* hist_out;
  const unsigned long long* R;
  const int2* items;
  const int* row_map;
  const float* VWh;           // kernel rows [rows][Q/2]
  const long long* ccdf;      // coarse CDF [rows][kCdfBlocks]
  const int* scale;           // fixed-point scale of each row
  const unsigned long long* thr_cell;
  const uint32_t* xlo;
  const uint32_t* xhi;
  uint4* pairs;               // queued events (id, cell, column, sign < 0)
  unsigned pair_cap;
  DevHeader* hdr;
  int n_x, n_M, Q, r0, child_wrap;
  uint32_t sim, k0, k1, t;
  int t_from_device;
  PhiloxKeys K;               // round keys of (k0, k1)
};

// p' of the pair created by particle id (column k, sign sgn) in cell c and the
// children c (k + M', +sgn), (k - M', -sgn); rows follow the cell index or the
// occupied list as the kernel stage laid them out.
template <bool SEQ = false>
__device__ __forceinline__ void pair_children(const StepArgs& a, int rows_by_cell, uint32_t id, uint32_t t, int c,
                                              int k, int sgn, unsigned long long& pairs, unsigned long long& dropped,
                                              long long& drop_signed) {
  const int n_M = a.n_M, h = a.Q / 2;
  const int orow = rows_by_cell ? c : __ldg(a.row_map + c);
  const uint4 wp = philox4x32_10k(make_uint4(id, t, kPurposePick, a.sim), a.K);
  const unsigned long long U2 = ((unsigned long long)(wp.x >> 5) << 26) | (unsigned long long)(wp.y >> 6);
  const float* vrow = a.VWh + (size_t)orow * h;
  const long long* crow = a.ccdf + (size_t)orow * kCdfBlocks;
  const int sc = __ldg(a.scale + orow);
  const int kp = SEQ ? sample_coarse_row_seq(vrow, crow, sc, a.Q, a.r0, n_M, U2)
                     : sample_coarse_row(vrow, crow, sc, a.Q, a.r0, n_M, U2);
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
    atomicAdd(a.hist_out + (size_t)c * n_M + kc, sc2[q]);
  }
}

// The same with the counters added to the header at once: the step kernel's
// rare path for events beyond the queue's capacity.
__device__ __forceinline__ void pair_children_direct(const StepArgs& a, int rows_by_cell, uint32_t id, uint32_t t,
                                                     int c, int k, int sgn) {
  unsigned long long pairs = 0, dropped = 0;
  long long drop_signed = 0;
  pair_children<true>(a, rows_by_cell, id, t, c, k, sgn, pairs, dropped, drop_signed);
  atomicAdd(&a.hdr->pairs, pairs);
  if (dropped) {
    atomicAdd(&a.hdr->dropped, dropped);
    atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->dropped_signed), (unsigned long long)drop_signed);
  }
}

// Sums five per-thread counters over the block into the header (one atomic each).
__device__ __forceinline__ void block_counters(DevHeader* hdr, unsigned long long pairs, unsigned long long absorbed,
                                               long long abs_signed, unsigned long long dropped,
                                               long long drop_signed) {
  __shared__ unsigned long long s_red[5][kStepWarps];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
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
  if (threadIdx.x < 5) {
    unsigned long long v = 0;
    for (int w = 0; w < kStepWarps; ++w) v += s_red[threadIdx.x][w];
    if (v) {
      unsigned long long* dst[5] = {&hdr->pairs, &hdr->absorbed, reinterpret_cast<unsigned long long*>(&hdr->absorbed_signed),
                                    &hdr->dropped, reinterpret_cast<unsigned long long*>(&hdr->dropped_signed)};
      atomicAdd(dst[threadIdx.x], v);
    }
  }
}

// Lane blocks of the staged row prefix: E2 = the power of two >= ceil(n_M / 32)
// columns per lane.
__host__ __device__ __forceinline__ int step_lg_block(int n_M) {
  int lg = 0;
  while ((32 << lg) < n_M) ++lg;
  return lg;
}

// Shared memory of a step block: the per-column move test (flip, threshold)
// of the block, then per warp the row prefix in a padded layout (column k at
// k + (k >> lg), so that lane l's block of E2 = 2^lg columns is contiguous and
// bank-conflict free), the sign bits, the non-empty bits and the event queue.
__host__ __device__ __forceinline__ int step_warp_words(int n_M) {
  const int E2 = 1 << step_lg_block(n_M);
  return 32 * (E2 + 1) + 1 + 2 * ((n_M + 31) / 32) + kPairQ;
}

static size_t step_smem(int n_M) {
  return sizeof(uint32_t) * (2 * (size_t)n_M + (size_t)kStepWarps * step_warp_words(n_M));
}

// 4-bit mask of the elements j of a quad with j < d (d may be <= 0 or >= 4).
__device__ __forceinline__ uint32_t first_mask(int d) { return d >= 4 ? 0xfu : (d <= 0 ? 0u : (1u << d) - 1u); }

__global__ __launch_bounds__(kStepThreads, 4) void k_step(StepArgs a) {
  extern __shared__ __align__(16) uint32_t smem_step[];
  __shared__ int s_qn[kStepWarps];
  __shared__ unsigned long long s_thr[kStepWarps][3];  // event thresholds of cells i - 1, i, i + 1
  const int n_M = a.n_M;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int lg = step_lg_block(n_M), E2 = 1 << lg;
  uint2* s_xm = reinterpret_cast<uint2*>(smem_step);
  uint32_t* wsm = smem_step + 2 * n_M + wid * step_warp_words(n_M);
  int* s_pp = reinterpret_cast<int*>(wsm);             // padded row prefix
  const int NW = (n_M + 31) / 32;
  uint32_t* s_sg = wsm + 32 * (E2 + 1) + 1;             // sign bits (1: negative)
  uint32_t* s_nz = s_sg + NW;                            // non-empty bits
  uint32_t* s_q = s_nz + NW;                              // event queue
  const int rows_by_cell = (int)a.hdr->rows_by_cell;
  const uint32_t t = a.t_from_device ? a.hdr->step : a.t;
  const int n_items = a.hdr->n_items;
  const unsigned int chunk = work_chunk(a.hdr);
  // move test of column k: moves iff (w ^ flip) > thr, i.e. w > xhi (rightward
  // drift), w < xlo (leftward, by complementing), never (thr = 2^32 - 1)
  for (int k = tid; k < n_M; k += kStepThreads) {
    const uint32_t lo = a.xlo[k], hi = a.xhi[k];
    s_xm[k] = hi != 0xffffffffu ? make_uint2(0u, hi) : (lo ? make_uint2(0xffffffffu, ~lo) : make_uint2(0u, 0xffffffffu));
  }
  if (lane == 0) s_qn[wid] = 0;
  __syncthreads();
  auto P = [&](int k) { return s_pp[k + (k >> lg)]; };
  // the first non-empty column after kk (n_M if none), from the non-empty bits
  auto next_nonempty = [&](int kk) -> int {
    int c = (kk + 1) >> 5;
    uint32_t w = c < NW ? s_nz[c] & (0xffffffffu << ((kk + 1) & 31)) : 0u;
    while (!w && ++c < NW) w = s_nz[c];
    return w ? (c << 5) + __ffs(w) - 1 : n_M;
  };

  int cur_i = -1;
  uint32_t base = 0u;
  bool need_gen = false, any_full = false;
  uint32_t rej = 0u;
  // event threshold of a stayer, thr(i), as u < thr <=> u < min(thr, 2^32 - 1) or thr >= 2^32
  uint32_t thr_st32 = 0u;
  bool all_st = false;

  int item = 0;
  if (lane == 0) item = (int)atomicAdd(&a.hdr->item_ticket, 1u);
  item = __shfl_sync(0xffffffffu, item, 0);
  while (item < n_items) {
    int nxt = 0;
    if (lane == 0) nxt = (int)atomicAdd(&a.hdr->item_ticket, 1u);  // consumed at the end of this item
    const int2 it = __ldg(a.items + item);
    const int i = it.x, ch = it.y;
    if (i != cur_i) {
      // stage the row: |n| into the padded buffer, sign bits, then the
      // exclusive prefix in place (lane l over its block of E2 columns)
      const int32_t* row = a.hist_in + (size_t)i * n_M;
      for (int k0 = 0; k0 < n_M; k0 += 32) {
        const int k = k0 + lane;
        const int n = k < n_M ? __ldg(row + k) : 0;
        if (k < n_M) s_pp[k + (k >> lg)] = n < 0 ? -n : n;
        const uint32_t b = __ballot_sync(0xffffffffu, n < 0);
        const uint32_t z = __ballot_sync(0xffffffffu, n != 0);
        if (lane == 0) {
          s_sg[k0 >> 5] = b;
          s_nz[k0 >> 5] = z;
        }
      }
      __syncwarp();
      const int kb0 = min(lane << lg, n_M), kb1 = min(kb0 + E2, n_M);
      int* blk = s_pp + lane * (E2 + 1);
      int local = 0;
      for (int j = 0; j < kb1 - kb0; ++j) local += blk[j];
      int incl = local;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += u;
      }
      int run = incl - local;
      for (int j = 0; j < kb1 - kb0; ++j) {
        const int v = blk[j];
        blk[j] = run;
        run += v;
      }
      __syncwarp();
      if (lane == 31) s_pp[n_M + (n_M >> lg)] = incl;
      base = (uint32_t)__ldg(a.R + i);
      const unsigned long long thr_m = i > 0 ? __ldg(a.thr_cell + i - 1) : 0ull;
      const unsigned long long thr_0 = __ldg(a.thr_cell + i);
      const unsigned long long thr_p = i + 1 < a.n_x ? __ldg(a.thr_cell + i + 1) : 0ull;
      if (lane == 0) {
        s_thr[wid][0] = thr_m;
        s_thr[wid][1] = thr_0;
        s_thr[wid][2] = thr_p;
      }
      need_gen = (thr_m | thr_0 | thr_p) != 0ull;
      all_st = (thr_0 >> 32) != 0ull;
      thr_st32 = all_st ? 0xffffffffu : (uint32_t)thr_0;
      // events: a stayer tests thr(i), a mover thr(i +- 1) (0 outside the
      // domain: absorbed particles create no pair); rej = the largest of them
      // as a quick rejection of a whole quad (exact unless a threshold is 2^32)
      const unsigned long long tmax =
          thr_0 > thr_m ? (thr_0 > thr_p ? thr_0 : thr_p) : (thr_m > thr_p ? thr_m : thr_p);
      any_full = tmax >> 32 != 0ull;
      rej = any_full ? 0xffffffffu : (uint32_t)tmax;
      cur_i = i;
      __syncwarp();
    }
    const uint32_t Ti = (uint32_t)P(n_M);
    // the item is [item0, item1) of the quad-aligned id range of the cell; each
    // lane takes a quad-aligned span of it
    const unsigned long long A = base & ~3u;
    const unsigned long long row_end = (unsigned long long)base + Ti;
    const unsigned long long item0 = A + (unsigned long long)ch * chunk;
    const unsigned long long item1 = item0 + chunk < row_end ? item0 + chunk : row_end;
    const uint32_t len = item1 > item0 ? (uint32_t)(item1 - item0) : 0u;
    const uint32_t span = ((len + 127u) >> 7) << 2;
    const unsigned long long lo64 = item0 + (unsigned long long)lane * span;
    const unsigned long long g0_64 = lo64 > base ? lo64 : base;
    const unsigned long long g1_64 = lo64 + span < item1 ? lo64 + span : item1;
    const bool has = g0_64 < g1_64;
    const uint32_t g0 = has ? (uint32_t)g0_64 : 0u, g1 = has ? (uint32_t)g1_64 : 0u;
    const uint32_t i0 = (uint32_t)item0;
    int32_t* const out_i = a.hist_out + (size_t)i * n_M;

    // bucket state
    int k = 0, sgn = 1, dir = 0;
    uint32_t end = 0u, flip = 0u, mthr = 0xffffffffu;
    uint32_t thr_mv32 = 0u;  // event threshold of a mover, thr(i + dir), in the same form
    bool all_mv = false;
    int n_st = 0, n_mv = 0;
    auto load_bucket = [&]() {
      end = base + (uint32_t)P(k + 1);
      sgn = ((s_sg[k >> 5] >> (k & 31)) & 1u) ? -1 : 1;
      const uint2 xm = s_xm[k];
      flip = xm.x;
      mthr = xm.y;
      dir = flip ? -1 : (mthr != 0xffffffffu ? 1 : 0);
      const unsigned long long thr_mv = s_thr[wid][dir + 1];
      all_mv = (thr_mv >> 32) != 0ull;
      thr_mv32 = all_mv ? 0xffffffffu : (uint32_t)thr_mv;
    };
    auto flush_bucket = [&]() {
      if (n_st) atomicAdd(out_i + k, sgn > 0 ? n_st : -n_st);
      if (n_mv) {
        const int c = sgn > 0 ? n_mv : -n_mv;
        if ((unsigned)(i + dir) < (unsigned)a.n_x) {
          atomicAdd(out_i + (dir > 0 ? n_M : -n_M) + k, c);
        } else {  // left the domain (edge cells only): counted at once
          atomicAdd(&a.hdr->absorbed, (unsigned long long)n_mv);
          atomicAdd(reinterpret_cast<unsigned long long*>(&a.hdr->absorbed_signed), (unsigned long long)(long long)c);
        }
      }
      n_st = n_mv = 0;
    };
    // pair event of particle id (mover or not) of the current bucket
    auto test_event = [&](uint32_t id, uint32_t u, int mv) {
      if (u < (mv ? thr_mv32 : thr_st32) || (mv ? all_mv : all_st)) {
        const int pos = atomicAdd(&s_qn[wid], 1);
        if (pos < kPairQ)  // always (the queue is drained whenever it could fill within one quad iteration)
          s_q[pos] = (id - i0) | ((uint32_t)k << 13) | ((uint32_t)(mv ? dir + 1 : 1) << 25) | (sgn < 0 ? 1u << 27 : 0u);
      }
    };
    // queued events of this item to the global queue (warp-collective)
    auto flush_queue = [&]() {
      __syncwarp();
      const int n = min(s_qn[wid], kPairQ);
      if (n) {
        unsigned qb = 0u;
        if (lane == 0) qb = atomicAdd(&a.hdr->pair_count, (unsigned)n);
        qb = __shfl_sync(0xffffffffu, qb, 0);
        for (int e = lane; e < n; e += 32) {
          const uint32_t q = s_q[e];
          const uint32_t id = i0 + (q & 8191u);
          const int kk = (int)((q >> 13) & 4095u), c = i - 1 + (int)((q >> 25) & 3u);
          const int sg = (q >> 27) & 1u ? -1 : 1;
          const unsigned slot = qb + (unsigned)e;
          if (slot >= qb && slot < a.pair_cap)
            a.pairs[slot] = make_uint4(id, (uint32_t)c, (uint32_t)kk, sg < 0 ? 1u : 0u);
          else
            pair_children_direct(a, rows_by_cell, id, t, c, kk, sg);
        }
        __syncwarp();
        if (lane == 0) s_qn[wid] = 0;
      }
      __syncwarp();
    };

    if (has) {
      // largest k with prefix(k) <= g0 - base: the bucket of the lane's first id
      const int lid = (int)(g0 - base);
      int lo = 0, hi = n_M;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (P(mid) <= lid) lo = mid; else hi = mid;
      }
      k = lo;
      load_bucket();
    }
    const int nq = (int)(span >> 2);
    const uint32_t q_first = (uint32_t)(lo64 >> 2);
#pragma unroll 1
    for (int jq = 0; jq < nq; ++jq) {
      const uint32_t q = q_first + (uint32_t)jq;
      const uint32_t qa = q << 2;
      if (qa < g1 && qa + 4u > g0) {  // (g0 = g1 = 0 for a lane without ids)
        uint4 wr = make_uint4(q, t - 1u, kPurposeRepos, a.sim);
        uint4 wg = make_uint4(q, t, kPurposeGen, a.sim);
        if (need_gen) philox4x32_10_x2k(wr, wg, a.K);
        else wr = philox4x32_10k(wr, a.K);
        const bool ev_possible = need_gen && (min(min(wg.x, wg.y), min(wg.z, wg.w)) < rej || any_full);
        // the ids of the quad in [g0, g1), bucket by bucket: the ids below the
        // current bucket's end are its members (a bucket ends exactly where the
        // next non-empty one starts), counted together from their move bits;
        // a lane whose quad crosses a bucket end takes a second pass
        uint32_t rem = 0xfu;
        if (qa < g0 || qa + 4u > g1) rem = first_mask((int)(g1 - qa)) & ~first_mask((int)(g0 - qa));
        const uint32_t w4[4] = {wr.x, wr.y, wr.z, wr.w};
        const uint32_t u4[4] = {wg.x, wg.y, wg.z, wg.w};
        while (true) {
          const uint32_t inb = rem & first_mask((int)(end - qa));
          uint32_t mvb = 0u;
#pragma unroll
          for (int j = 0; j < 4; ++j) mvb |= (uint32_t)((w4[j] ^ flip) > mthr) << j;
          mvb &= inb;
          const int m = __popc(mvb);
          n_mv += m;
          n_st += __popc(inb) - m;
          if (ev_possible) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
              if ((inb >> j) & 1u) test_event(qa + (uint32_t)j, u4[j], (int)((mvb >> j) & 1u));
          }
          rem &= ~inb;
          if (!rem) break;
          flush_bucket();
          k = next_nonempty(k);
          load_bucket();
        }
      }
      __syncwarp();
      if (s_qn[wid] > kPairQ - 128) flush_queue();
    }
    if (has) flush_bucket();
    flush_queue();
    item = __shfl_sync(0xffffffffu, nxt, 0);
  }
  if (blockIdx.x == 0 && tid == 0 && n_items > 0) atomicAdd(&a.hdr->particle_steps, a.hdr->population);
}

// The queued pair events of the step: one thread each.  The last block to
// finish resets the queue and the work-item ticket for the next step.
__global__ __launch_bounds__(kStepThreads) void k_pairs(StepArgs a) {
  const int rows_by_cell = (int)a.hdr->rows_by_cell;
  const uint32_t t = a.t_from_device ? a.hdr->step : a.t;
  const unsigned cnt = a.hdr->pair_count;
  const unsigned n = cnt < a.pair_cap ? cnt : a.pair_cap;
  unsigned long long pairs = 0, dropped = 0;
  long long drop_signed = 0;
  for (unsigned e = blockIdx.x * kStepThreads + threadIdx.x; e < n; e += gridDim.x * kStepThreads) {
    const uint4 ev = a.pairs[e];
    pair_children(a, rows_by_cell, ev.x, t, (int)ev.y, (int)ev.z, ev.w ? -1 : 1, pairs, dropped, drop_signed);
  }
  block_counters(a.hdr, pairs, 0ull, 0ll, dropped, drop_signed);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&a.hdr->pairs_done, 1u) == gridDim.x - 1u) {
      a.hdr->pair_count = 0u;
      a.hdr->item_ticket = 0u;
      a.hdr->chunk = a.hdr->chunk_next ? a.hdr->chunk_next : (unsigned int)kChunk;
      a.hdr->pairs_done = 0u;
      __threadfence();
    }
  }
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
  if (sm > 48 * 1024) raise_smem_limit(reinterpret_cast<const void*>(k_step), sm);
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
  const Layout L = layout(p);
  StepArgs a;
  a.hist_in = hist_in;
  a.hist_out = hist_out;
  a.R = v.R;
  a.items = v.items;
  a.row_map = v.row_map;
  a.VWh = v.VWh;
  a.ccdf = v.ccdf;
  a.scale = v.scale;
  a.thr_cell = v.thr_cell;
  a.xlo = v.xlo;
  a.xhi = v.xhi;
  a.pairs = v.pairs;
  a.pair_cap = L.pair_cap;
  a.hdr = v.hdr;
  a.n_x = p.n_x;
  a.n_M = p.n_M;
  a.Q = p.Q;
  a.r0 = ((-(p.n_M / 2)) % p.Q + p.Q) % p.Q;
  a.child_wrap = p.child_wrap;
  a.sim = p.sim;
  a.k0 = (uint32_t)(p.seed & 0xffffffffu);
  a.k1 = (uint32_t)(p.seed >> 32);
  a.K = philox_keys(a.k0, a.k1);
  a.t = t;
  a.t_from_device = t_from_device;
  const int grid = step_grid(p.n_M);
  cudaError_t e = step_timing_record(s, false);
  if (e != cudaSuccess) return e;
  k_step<<<grid, kStepThreads, step_smem(p.n_M), s>>>(a);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = step_timing_record(s, true);
  if (e != cudaSuccess) return e;
  // one thread per queued event (the count is on the device: surplus blocks exit)
  const unsigned pair_blocks = (L.pair_cap + kStepThreads - 1) / kStepThreads;
  k_pairs<<<pair_blocks < 8u * (unsigned)num_sms() ? pair_blocks : 8u * (unsigned)num_sms(), kStepThreads, 0, s>>>(a);
  return cudaGetLastError();
}

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
  const unsigned long long id_base = hdr->id_base;
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
    const int per_item = (int)work_chunk(hdr), kPer = per_item / kStepThreads;
    const int lo = chunk * per_item + tid * kPer;  // ids [chunk c, (chunk + 1) c) of the row, c ids per item
    const int hi = min(lo + kPer, Ti);
    if (lo < hi) {
      int k = bucket_of(s_pre, n_M, lo);
      for (int lid = lo; lid < hi; ++lid) {
        while (s_pre[k + 1] <= lid) ++k;
        const uint32_t id = base + (uint32_t)lid;
        const uint4 w = philox4x32_10(make_uint4(id >> 2, t, kPurposeRepos, sim), k0, k1);
        const uint32_t wj = (id & 3u) == 0u ? w.x : ((id & 3u) == 1u ? w.y : ((id & 3u) == 2u ? w.z : w.w));
        const uint32_t o = id - (uint32_t)id_base;  // place in this histogram
        cell[o] = i;
        f[o] = (float)(wj >> 8) * 0x1p-24f;
        M[o] = (int16_t)(k - n_M / 2);
        sign[o] = (int8_t)(s_n[k] > 0 ? 1 : -1);
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
