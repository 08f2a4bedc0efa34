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
// (Sec. 2.2).
__global__ void k_init_tables(int n_M, int Q, double d1, float* __restrict__ D, uint32_t* __restrict__ xlo,
                              uint32_t* __restrict__ xhi, float* __restrict__ B, int Kp, int Np, DevHeader* hdr) {
  const int h = Q / 2;
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
  for (long long q = tid; q < (long long)Kp * Np; q += nthreads) {
    const int kk = (int)(q / Np), r = (int)(q % Np);
    float v = 0.f;
    if (kk < h - 1 && r < h) {
      const long long t = ((long long)(kk + 1) * r) % Q;
      v = __double2float_rn(sinpi(2.0 * (double)t / (double)Q));
    }
    B[q] = v;
  }
}

cudaError_t launch_init_tables(const wmc_params& p, const View& v, cudaStream_t s) {
  const Layout L = layout(p);
  const double d1 = ((kHbarJs * kPi) * p.dt_s) / ((p.mass_kg * (double)p.Q) * (p.dx_m * p.dx_m));
  k_init_tables<<<256, 256, 0, s>>>(p.n_M, p.Q, d1, v.D, v.xlo, v.xhi, v.B, L.Kp, L.Np, v.hdr);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- per-cell scan and plan

// T and reach of every cell staged in shared memory by coalesced loads when
// they fit, so the scan's per-thread runs read on-chip memory
constexpr int kPlanStage = 4096;

// The plan, by one block (blockDim.x threads, a multiple of 32 up to 1024):
// exclusive prefix sums of survivors (ids), work items and needed cells, then
// the occupied list, row map and work-item descriptors; with clear_thr the
// per-cell event thresholds are cleared (a kernel stage over the occupied list
// then fills the occupied cells; one over every cell writes them all itself).
__device__ __forceinline__ void plan_block(int n_x, const unsigned long long* T_g, const unsigned char* reach_g,
                           unsigned long long* __restrict__ R, int* __restrict__ IP, int* __restrict__ occ,
                           int* __restrict__ row_map, int2* __restrict__ items, long long max_items,
                           unsigned long long* __restrict__ thr_cell, DevHeader* hdr, int advance_step,
                           int clear_thr) {
  __shared__ unsigned long long wT[32];
  __shared__ int wI[32], wN[32], wBig[32];
  __shared__ unsigned long long s_T[kPlanStage];
  __shared__ unsigned char s_reach[kPlanStage];
  const int nt = blockDim.x, nw = nt >> 5;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const unsigned long long* T = T_g;
  const unsigned char* reach = reach_g;
  if (n_x <= kPlanStage) {
    for (int i = tid; i < n_x; i += nt) {
      s_T[i] = __ldg(T_g + i);
      s_reach[i] = __ldg(reach_g + i);
    }
    __syncthreads();
    T = s_T;
    reach = s_reach;
  }
  const int per = (n_x + nt - 1) / nt;
  const int lo = min(tid * per, n_x), hi = min(lo + per, n_x);
  unsigned long long aT = 0;
  int aI = 0, aN = 0, big = 0;
  for (int i = lo; i < hi; ++i) {
    const unsigned long long t = T[i];
    aT += t;
    aI += items_of_cell(t);
    aN += cell_needs_kernel(reach, i, n_x);
    big |= t > 0x7fffffffull;
  }
  // block-wide exclusive scan of (aT, aI, aN)
  unsigned long long iT = aT;
  int iI = aI, iN = aN;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned long long uT = __shfl_up_sync(0xffffffffu, iT, off);
    const int uI = __shfl_up_sync(0xffffffffu, iI, off);
    const int uN = __shfl_up_sync(0xffffffffu, iN, off);
    if (lane >= off) {
      iT += uT;
      iI += uI;
      iN += uN;
    }
  }
  big = __any_sync(0xffffffffu, big);
  if (lane == 31) {
    wT[wid] = iT;
    wI[wid] = iI;
    wN[wid] = iN;
    wBig[wid] = big;
  }
  __syncthreads();
  if (wid == 0) {
    unsigned long long sT = lane < nw ? wT[lane] : 0ull;
    int sI = lane < nw ? wI[lane] : 0, sN = lane < nw ? wN[lane] : 0, sB = lane < nw ? wBig[lane] : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned long long uT = __shfl_up_sync(0xffffffffu, sT, off);
      const int uI = __shfl_up_sync(0xffffffffu, sI, off);
      const int uN = __shfl_up_sync(0xffffffffu, sN, off);
      if (lane >= off) {
        sT += uT;
        sI += uI;
        sN += uN;
      }
    }
    sB = __any_sync(0xffffffffu, sB);
    wT[lane] = sT;
    wI[lane] = sI;
    wN[lane] = sN;
    wBig[lane] = sB;
  }
  __syncthreads();
  const unsigned long long baseT = (wid ? wT[wid - 1] : 0ull) + iT - aT;
  int baseI = (wid ? wI[wid - 1] : 0) + iI - aI;
  int baseN = (wid ? wN[wid - 1] : 0) + iN - aN;
  const int ok = !wBig[31] && wT[31] < (1ull << 32) && (long long)wI[31] <= max_items;
  unsigned long long r = baseT;
  for (int i = lo; i < hi; ++i) {
    const unsigned long long t = T[i];
    if (ok) {
      const int ni = items_of_cell(t);
      for (int c = 0; c < ni; ++c) items[baseI + c] = make_int2(i, c);
    }
    if (clear_thr) thr_cell[i] = 0ull;
    R[i] = r;
    IP[i] = baseI;
    if (cell_needs_kernel(reach, i, n_x)) {
      occ[baseN] = i;
      row_map[i] = baseN;
      ++baseN;
    } else {
      row_map[i] = -1;
    }
    r += t;
    baseI += items_of_cell(t);
  }
  if (tid == nt - 1) {
    const unsigned long long P = wT[31];
    const int too_big = !ok;
    R[n_x] = P;
    IP[n_x] = wI[31];
    hdr->population = P;
    hdr->n_items = too_big ? 0 : wI[31];
    hdr->n_occ = wN[31];
    if (too_big) atomicOr(&hdr->flags, WMC_FLAG_CAPACITY);
    if (advance_step) hdr->step += 1u;
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

// The plan as its own single-block launch (n_x is at most a few 10^4 in the
// workloads and this runs once per step).
constexpr int kPlanThreads = 1024;

__global__ __launch_bounds__(kPlanThreads) void k_plan(int n_x, const unsigned long long* __restrict__ T,
                                                       const unsigned char* __restrict__ reach,
                                                       unsigned long long* __restrict__ R, int* __restrict__ IP,
                                                       int* __restrict__ occ, int* __restrict__ row_map,
                                                       int2* __restrict__ items, long long max_items,
                                                       unsigned long long* __restrict__ thr_cell, DevHeader* hdr,
                                                       int advance_step, int clear_thr) {
  plan_block(n_x, T, reach, R, IP, occ, row_map, items, max_items, thr_cell, hdr, advance_step, clear_thr);
}

cudaError_t launch_rows(const wmc_params& p, const View& v, const int32_t* hist, int64_t* rho, cudaStream_t s,
                        int32_t* zero_out) {
  const int blocks = (p.n_x + kRowsWarps - 1) / kRowsWarps;
  k_rows<<<blocks, kRowsWarps * 32, 0, s>>>(hist, p.n_x, p.n_M, v.D, v.T, v.reach,
                                            reinterpret_cast<long long*>(rho), zero_out);
  return cudaGetLastError();
}

cudaError_t launch_plan_scan(const wmc_params& p, const View& v, int advance_step, int clear_thr, cudaStream_t s) {
  k_plan<<<1, kPlanThreads, 0, s>>>(p.n_x, v.T, v.reach, v.R, v.IP, v.occ, v.row_map, v.items,
                                    layout(p).max_items, v.thr_cell, v.hdr, advance_step, clear_thr);
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

cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, long long n, uint32_t* out,
                          cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long long blocks = (n + 255) / 256;
  k_philox<<<(unsigned)(blocks < 65535 ? blocks : 65535), 256, 0, s>>>(reinterpret_cast<const uint4*>(ctr), k0, k1,
                                                                      n, reinterpret_cast<uint4*>(out));
  return cudaGetLastError();
}

}  // namespace wmc
