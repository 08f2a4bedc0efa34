// Survivor enumeration after annihilation (rule 2), occupied cells for the
// kernel, density (rule 1), constant tables and the Philox check kernel.
#include <math.h>

#include "wmc_device.cuh"

namespace wmc {

// ---------------------------------------------------------------- constant tables
// D[k] = fl32(M * d1), d1 = hbar pi dt / (m Q dx^2), M = k - n_M/2: the free
// drift of momentum M dp over dt, in cells.  Crossing thresholds on the offset
// word w (f = (w >> 8) 2^-24): a particle of column k moves right iff
// fl32(f + D) >= 1 iff w > xhi[k], left iff fl32(f + D) < 0 iff w < xlo[k].
// B[kk][r] = sin(2 pi ((kk+1) r mod Q) / Q) for kk < h-1, r < h (zero padding
// elsewhere): the integer-indexed sine matrix of the network's hidden layer
// (Sec. 2.2); B2[u][r] the folded matrix of the N = 2 network (Sec. 2.3).
__global__ void k_init_tables(int n_M, int Q, double d1, float* __restrict__ D, uint32_t* __restrict__ xlo,
                              uint32_t* __restrict__ xhi, float* __restrict__ B, int Kp, int Np,
                              float* __restrict__ B2, int Kp2, DevHeader* hdr) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  if (tid == 0) {
    DevHeader z = {};
    z.magic = kMagic;
    *hdr = z;
  }
  for (long long k = tid; k < n_M; k += nthreads) {
    const float d = __double2float_rn((double)(k - n_M / 2) * d1);
    D[k] = d;
    uint32_t lo = 0u, hi = 0xffffffffu;
    if (d > 0.f) hi = (uint32_t)(((unsigned long long)first_offset_reaching(d, 1.f) << 8) - 1ull);
    if (d < 0.f) lo = (uint32_t)((unsigned long long)first_offset_reaching(d, 0.f) << 8);
    xlo[k] = lo;
    xhi[k] = hi;
  }
  for (long long q = tid; q < (long long)Kp * Np; q += nthreads) B[q] = sine_entry_n1(Q, (int)(q / Np), (int)(q % Np));
  for (long long q = tid; q < (long long)Kp2 * Np; q += nthreads) B2[q] = sine_entry_n2(Q, (int)(q / Np), (int)(q % Np));
}

cudaError_t launch_init_tables(const wmc_params& p, const View& v, cudaStream_t s) {
  const Layout L = layout(p);
  const double d1 = ((kHbarJs * kPi) * p.dt_s) / ((p.mass_kg * (double)p.Q) * (p.dx_m * p.dx_m));
  k_init_tables<<<256, 256, 0, s>>>(p.n_M, p.Q, d1, v.D, v.xlo, v.xhi, v.B, L.Kp, L.Np, v.B2, L.Kp2, v.hdr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // no stale publication may carry a tag of a coming plan launch
  return cudaMemsetAsync(v.plan, 0, sizeof(PlanStatus) * (size_t)((p.n_x + kPlanCells - 1) / kPlanCells), s);
}

// ---------------------------------------------------------------- per-cell scan and plan
// The plan: exclusive prefix sums over the cells of survivors (the first id
// R[i] of each cell), work items (the first item IP[i]) and needed cells (the
// occupied list and its row map), then the item descriptors; with clear_thr
// the per-cell event thresholds are cleared (a kernel stage over the occupied
// list then fills the occupied cells).  One thread per cell, kPlanCells cells
// per block; the blocks chain their prefixes by a decoupled look-back: each
// publishes its own totals at once and its inclusive prefix as soon as it
// knows it, and a block sums its predecessors' totals back to the first
// inclusive prefix it meets.  Blocks take their logical index from a ticket,
// so every block waits only on blocks already running; every wait is bounded
// and a timeout sets WMC_FLAG_TIMEOUT.  The last block writes the totals to
// the header, resets the ticket and advances the epoch that tags the
// publications.
constexpr long long kPlanWaitCycles = 2000000000ll;

__device__ __forceinline__ PlanSums plan_add(const PlanSums& a, const PlanSums& b) {
  PlanSums r;
  r.T = a.T + b.T;
  r.I = a.I + b.I;
  r.N = a.N + b.N;
  r.big = a.big | b.big;
  r.pad = 0;
  return r;
}

__device__ __forceinline__ PlanSums plan_load(const volatile PlanSums* p) {
  PlanSums r;
  r.T = p->T;
  r.I = p->I;
  r.N = p->N;
  r.big = p->big;
  r.pad = 0;
  return r;
}

__device__ __forceinline__ void plan_store(volatile PlanSums* p, const PlanSums& v) {
  p->T = v.T;
  p->I = v.I;
  p->N = v.N;
  p->big = v.big;
}

__global__ __launch_bounds__(kPlanCells) void k_plan(int n_x, const unsigned long long* __restrict__ T,
                                                     const unsigned char* __restrict__ reach,
                                                     unsigned long long* __restrict__ R, int* __restrict__ IP,
                                                     int* __restrict__ occ, int* __restrict__ row_map,
                                                     int2* __restrict__ items, long long max_items,
                                                     unsigned long long* __restrict__ thr_cell, DevHeader* hdr,
                                                     PlanStatus* st, int advance_step, int clear_thr, int step_warps) {
  __shared__ PlanSums w_s[kPlanCells / 32];
  __shared__ PlanSums s_ex;
  __shared__ int s_blk;
  __shared__ unsigned int s_epoch;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) {
    s_blk = (int)atomicAdd(&hdr->plan_ticket, 1u);
    s_epoch = *(volatile unsigned int*)&hdr->plan_epoch;
  }
  __syncthreads();
  const int blk = s_blk;
  const unsigned int epoch = s_epoch;
  const int i = blk * kPlanCells + tid;
  const unsigned long long t = i < n_x ? __ldg(T + i) : 0ull;
  const unsigned int chunk = work_chunk(hdr);  // (changed only after the step, by the pair kernel)
  PlanSums mine;
  mine.T = t;
  mine.I = items_of_cell(t, chunk);
  mine.N = i < n_x ? cell_needs_kernel(reach, i, n_x) : 0;
  mine.big = t > 0x7fffffffull;
  mine.pad = 0;
  // block-wide inclusive scan
  PlanSums inc = mine;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    PlanSums u;
    u.T = __shfl_up_sync(0xffffffffu, inc.T, off);
    u.I = __shfl_up_sync(0xffffffffu, inc.I, off);
    u.N = __shfl_up_sync(0xffffffffu, inc.N, off);
    u.big = __shfl_up_sync(0xffffffffu, inc.big, off);
    if (lane >= off) inc = plan_add(inc, u);
  }
  if (lane == 31) w_s[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    PlanSums w = w_s[lane];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      PlanSums u;
      u.T = __shfl_up_sync(0xffffffffu, w.T, off);
      u.I = __shfl_up_sync(0xffffffffu, w.I, off);
      u.N = __shfl_up_sync(0xffffffffu, w.N, off);
      u.big = __shfl_up_sync(0xffffffffu, w.big, off);
      if (lane >= off) w = plan_add(w, u);
    }
    w_s[lane] = w;
  }
  __syncthreads();
  if (wid) inc = plan_add(inc, w_s[wid - 1]);
  const PlanSums agg = w_s[kPlanCells / 32 - 1];
  // look-back by warp 0: lane l inspects predecessor blk - 1 - l - 32 w of
  // window w, waiting (bounded) until it has published; the nearest inclusive
  // prefix ends the walk, aggregates before it are added
  if (wid == 0) {
    volatile PlanStatus* me = st + blk;
    if (lane == 0) {
      plan_store(&me->agg, agg);
      if (blk == 0) plan_store(&me->inc, agg);
      __threadfence();
      me->tag = (epoch << 2) | (blk == 0 ? 2u : 1u);
    }
    PlanSums ex = {0ull, 0, 0, 0, 0};
    bool timed_out = false;
    for (int top = blk - 1; top >= 0 && !timed_out; top -= 32) {
      const int j = top - lane;
      unsigned int tag = (epoch << 2) | 1u;
      if (j >= 0) {
        const volatile PlanStatus* o = st + j;
        const long long t0 = clock64();
        while (((tag = o->tag) >> 2) != (epoch & 0x3fffffffu) || (tag & 3u) == 0u) {
          if (clock64() - t0 > kPlanWaitCycles) {
            timed_out = true;
            break;
          }
          __nanosleep(32);
        }
      }
      timed_out = __any_sync(0xffffffffu, timed_out);
      if (timed_out) break;
      __threadfence();
      const unsigned incl = __ballot_sync(0xffffffffu, j >= 0 && (tag & 3u) == 2u);
      const int stop = incl ? __ffs(incl) - 1 : 32;   // nearest inclusive prefix in this window
      PlanSums mineb = {0ull, 0, 0, 0, 0};
      if (j >= 0 && lane <= stop) mineb = lane == stop ? plan_load(&st[j].inc) : plan_load(&st[j].agg);
#pragma unroll
      for (int off = 16; off; off >>= 1) {
        PlanSums u;
        u.T = __shfl_down_sync(0xffffffffu, mineb.T, off);
        u.I = __shfl_down_sync(0xffffffffu, mineb.I, off);
        u.N = __shfl_down_sync(0xffffffffu, mineb.N, off);
        u.big = __shfl_down_sync(0xffffffffu, mineb.big, off);
        mineb = plan_add(mineb, u);
      }
      ex = plan_add(ex, mineb);  // (lane 0 holds the window's sum)
      if (incl) break;
    }
    if (lane == 0) {
      if (timed_out) atomicOr(&hdr->flags, WMC_FLAG_TIMEOUT);
      if (blk > 0) {
        plan_store(&me->inc, plan_add(ex, agg));
        __threadfence();
        me->tag = (epoch << 2) | 2u;
      }
      s_ex = ex;
    }
  }
  __syncthreads();
  const PlanSums ex = s_ex;
  const PlanSums tot = plan_add(ex, agg);  // through the block's last cell
  const unsigned long long id_base = hdr->id_base;
  if (i < n_x) {
    const unsigned long long r = id_base + ex.T + inc.T - mine.T;
    const int baseI = ex.I + inc.I - mine.I;
    const int baseN = ex.N + inc.N - mine.N;
    R[i] = r;
    IP[i] = baseI;
    for (int c = 0; c < mine.I; ++c)
      if ((long long)baseI + c < max_items) items[baseI + c] = make_int2(i, c);
    if (clear_thr) thr_cell[i] = 0ull;
    if (mine.N) {
      occ[baseN] = i;
      row_map[i] = baseN;
    } else {
      row_map[i] = -1;
    }
  }
  if (blk == (int)gridDim.x - 1 && tid == 0) {
    // totals of every cell
    const bool ok = !tot.big && id_base + tot.T < (1ull << 32) && (long long)tot.I <= max_items;
    R[n_x] = id_base + tot.T;
    IP[n_x] = tot.I;
    hdr->population = tot.T;
    hdr->n_items = ok ? tot.I : 0;
    hdr->n_occ = tot.N;
    if (!ok) atomicOr(&hdr->flags, WMC_FLAG_CAPACITY);
    if (advance_step) hdr->step += 1u;
    // items for the next step: about four per step warp at this population,
    // at least kMinChunk ids, at most kChunk (work distribution only: results
    // do not depend on it)
    {
      const unsigned long long per = tot.T / (4ull * (unsigned long long)(step_warps > 0 ? step_warps : 1));
      unsigned int c = kMinChunk;
      while (c < per && c < (unsigned int)kChunk) c <<= 1;
      hdr->chunk_next = c;
    }
    hdr->plan_ticket = 0u;
    hdr->plan_epoch = (epoch + 1u) & 0x3fffffffu;
    __threadfence();
  }
}

// One warp per cell: survivors T[i] = sum_k |n(i,k)|, reach bits (bit0 cell
// occupied, bit1 a momentum that drifts right is present, bit2 one that drifts
// left), optionally the density rho[i] = sum_k n(i,k), and optionally a zeroed
// row of the next histogram.
constexpr int kRowsWarps = 8;

__global__ __launch_bounds__(kRowsWarps * 32) void k_rows(const int32_t* __restrict__ hist, int n_x, int n_M,
                                                          const float* __restrict__ D,
                                                          unsigned long long* __restrict__ T,
                                                          unsigned char* __restrict__ reach,
                                                          long long* __restrict__ rho, int32_t* __restrict__ zero_out) {
  const int warp = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp < n_x) {
    const int32_t* row = hist + (size_t)warp * n_M;
    unsigned long long a = 0;
    long long sn = 0;
    unsigned bits = 0;
    if ((n_M & 3) == 0) {
      const int4* row4 = reinterpret_cast<const int4*>(row);
      const float4* D4 = reinterpret_cast<const float4*>(D);
      int4* z4 = zero_out ? reinterpret_cast<int4*>(zero_out + (size_t)warp * n_M) : nullptr;
      for (int q = lane; q < n_M / 4; q += 32) {
        const int4 n = row4[q];
        const float4 d = D4[q];
        if (z4) z4[q] = make_int4(0, 0, 0, 0);
        const int nv[4] = {n.x, n.y, n.z, n.w};
        const float dv[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (nv[e]) {
            a += (unsigned long long)(nv[e] < 0 ? -(long long)nv[e] : (long long)nv[e]);
            sn += nv[e];
            bits |= 1u | (dv[e] > 0.f ? 2u : 0u) | (dv[e] < 0.f ? 4u : 0u);
          }
        }
      }
    } else {
      for (int k = lane; k < n_M; k += 32) {
        const int n = row[k];
        if (zero_out) zero_out[(size_t)warp * n_M + k] = 0;
        if (n) {
          a += (unsigned long long)(n < 0 ? -(long long)n : (long long)n);
          sn += n;
          bits |= 1u | (D[k] > 0.f ? 2u : 0u) | (D[k] < 0.f ? 4u : 0u);
        }
      }
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, off);
      sn += __shfl_down_sync(0xffffffffu, sn, off);
      bits |= __shfl_down_sync(0xffffffffu, bits, off);
    }
    if (lane == 0) {
      T[warp] = a;
      reach[warp] = (unsigned char)bits;
      if (rho) rho[warp] = sn;
    }
  }
}

cudaError_t launch_rows(const wmc_params& p, const View& v, const int32_t* hist, int64_t* rho, cudaStream_t s,
                        int32_t* zero_out) {
  const int blocks = (p.n_x + kRowsWarps - 1) / kRowsWarps;
  k_rows<<<blocks, kRowsWarps * 32, 0, s>>>(hist, p.n_x, p.n_M, v.D, v.T, v.reach,
                                            reinterpret_cast<long long*>(rho), zero_out);
  return cudaGetLastError();
}

cudaError_t launch_plan_scan(const wmc_params& p, const View& v, int advance_step, int clear_thr, cudaStream_t s) {
  const int blocks = (p.n_x + kPlanCells - 1) / kPlanCells;
  k_plan<<<blocks, kPlanCells, 0, s>>>(p.n_x, v.T, v.reach, v.R, v.IP, v.occ, v.row_map, v.items,
                                       layout(p).max_items, v.thr_cell, v.hdr, v.plan, advance_step, clear_thr,
                                       step_grid(p.n_M) * kStepWarps);
  return cudaGetLastError();
}

cudaError_t launch_plan(const wmc_params& p, const View& v, const int32_t* hist, int64_t* rho, int advance_step,
                        cudaStream_t s, int32_t* zero_out) {
  cudaError_t e = launch_rows(p, v, hist, rho, s, zero_out);
  if (e != cudaSuccess) return e;
  return launch_plan_scan(p, v, advance_step, 1, s);
}

// ---------------------------------------------------------------- density
__global__ void k_density(const int32_t* __restrict__ hist, int n_x, int n_M, long long* __restrict__ rho) {
  const int warp = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= n_x) return;
  const int32_t* row = hist + (size_t)warp * n_M;
  long long sn = 0;
  for (int k = lane; k < n_M; k += 32) sn += row[k];
#pragma unroll
  for (int off = 16; off; off >>= 1) sn += __shfl_down_sync(0xffffffffu, sn, off);
  if (lane == 0) rho[warp] = sn;
}

cudaError_t launch_density(const wmc_params& p, const int32_t* hist, int64_t* rho, cudaStream_t s) {
  const int blocks = (p.n_x + 7) / 8;
  k_density<<<blocks, 256, 0, s>>>(hist, p.n_x, p.n_M, reinterpret_cast<long long*>(rho));
  return cudaGetLastError();
}

// ---------------------------------------------------------------- Philox check
__global__ void k_philox(const uint4* __restrict__ ctr, uint32_t k0, uint32_t k1, long long n, uint4* __restrict__ out) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    out[q] = philox4x32_10(ctr[q], k0, k1);
}

// Throughput of the generator as the particle step uses it: each thread
// evaluates calls in pairs under one key schedule (counters (q, 1, 2, 0) and
// (q, 2, 1, 0) for distinct q) and folds every word into one XOR, written
// out so that no evaluation can be dropped.
__global__ __launch_bounds__(256) void k_philox_throughput(uint32_t k0, uint32_t k1, int pairs_per_thread,
                                                           uint32_t* __restrict__ out) {
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  uint32_t acc = 0u;
  for (int j = 0; j < pairs_per_thread; ++j) {
    const uint32_t q = g + (uint32_t)j * gs;
    uint4 a = make_uint4(q, 1u, 2u, 0u), b = make_uint4(q, 2u, 1u, 0u);
    philox4x32_10_x2(a, b, k0, k1);
    acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w;
  }
  out[g] = acc;
}

cudaError_t launch_philox_throughput(uint32_t k0, uint32_t k1, int pairs_per_thread, uint32_t* out, long long n_threads,
                                     cudaStream_t s) {
  k_philox_throughput<<<(unsigned)(n_threads / 256), 256, 0, s>>>(k0, k1, pairs_per_thread, out);
  return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, long long n, uint32_t* out,
                          cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long long blocks = (n + 255) / 256;
  k_philox<<<(unsigned)(blocks < 65535 ? blocks : 65535), 256, 0, s>>>(reinterpret_cast<const uint4*>(ctr), k0, k1,
                                                                      n, reinterpret_cast<uint4*>(out));
  return cudaGetLastError();
}

}  // namespace wmc
