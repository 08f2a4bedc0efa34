// One step of the postulate (Sec. 2.1) over the survivors of a net histogram:
// free drift, absorption, pair creation with probability gamma dt and momentum
// p' ~ V_W^+ / gamma, and the signed histogram of parents and children (whose
// summation is the annihilation of rule 2).
//
// The survivors are never stored: after annihilation every particle of bucket
// (i, M) carries the same cell, momentum and sign, and its offset is a Philox
// draw of its id, so the histogram and the id prefix describe the ensemble
// exactly.  A block takes a work item (up to kChunk consecutive ids of one
// cell), privatises the three histogram rows its particles can land in
// (i-1, i, i+1) in shared memory, and flushes them with one global atomic per
// non-zero bucket.
#include "wmc_internal.cuh"

namespace wmc {

struct StepArgs {
  const int32_t* hist_in;
  int32_t* hist_out;
  const unsigned long long* R;
  const int* IP;
  const int* row_map;
  const double* cdf;  // [n_M][ld]
  long long ld;
  const double* gamma;
  const unsigned long long* gthr;
  const float* D;
  const float* VWh;
  DevHeader* hdr;
  int n_x, n_M, Q, child_wrap;
  uint32_t sim, k0, k1, t;
  int t_from_device;
};

// Loads the signed counts of cell i into s_n and their exclusive prefix of
// |n| into s_pre[0..n_M] (s_pre[n_M] = survivors of the cell).
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

// Largest k with s_pre[k] <= lid (so s_pre[k] <= lid < s_pre[k+1]).
__device__ __forceinline__ int bucket_of(const int* s_pre, int n_M, int lid) {
  int lo = 0, hi = n_M;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (s_pre[mid] <= lid) lo = mid; else hi = mid;
  }
  return lo;
}

// V_W(row; M = k - n_M/2) from a half-period row.
__device__ __forceinline__ float kernel_at(const float* __restrict__ v, int Q, int n_M, int k) {
  const int h = Q / 2;
  int r = (k - n_M / 2) % Q;
  if (r < 0) r += Q;
  if (r == 0 || r == h) return 0.f;
  return r < h ? __ldg(v + r) : -__ldg(v + (Q - r));
}

// Index of p': the smallest k with cdf[k] > target, else the largest k with
// V_W^+ > 0 (a target equal to gamma after rounding).
__device__ __forceinline__ int sample_momentum(const StepArgs& a, int orow, double target) {
  const double* c = a.cdf + orow;
  int lo = 0, hi = a.n_M;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(c + (long long)mid * a.ld) > target) hi = mid; else lo = mid + 1;
  }
  if (lo < a.n_M) return lo;
  const float* v = a.VWh + (size_t)orow * (a.Q / 2);
  for (int k = a.n_M - 1; k >= 0; --k)
    if (kernel_at(v, a.Q, a.n_M, k) > 0.f) return k;
  return -1;
}

__global__ __launch_bounds__(kStepThreads) void k_step(StepArgs a) {
  extern __shared__ int smem[];
  const int n_M = a.n_M;
  int* s_pre = smem;                 // n_M + 1
  int* s_n = s_pre + (n_M + 1);      // n_M
  int* s_acc = s_n + n_M;            // 3 n_M: rows i-1, i, i+1
  float* s_D = reinterpret_cast<float*>(s_acc + 3 * n_M);  // n_M
  __shared__ int s_wsum[kStepThreads / 32];
  __shared__ int s_row;
  __shared__ unsigned long long s_red[5][kStepThreads / 32];

  const int tid = threadIdx.x;
  const uint32_t t = a.t_from_device ? a.hdr->step : a.t;
  const int n_items = a.hdr->n_items;
  for (int k = tid; k < n_M; k += kStepThreads) s_D[k] = a.D[k];

  unsigned long long pairs = 0, absorbed = 0, dropped = 0;
  long long abs_signed = 0, drop_signed = 0;

  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    __syncthreads();  // previous item fully flushed
    if (tid == 0) {
      int lo = 0, hi = a.n_x;  // largest i with IP[i] <= item
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(a.IP + mid) <= item) lo = mid; else hi = mid;
      }
      s_row = lo;
    }
    for (int q = tid; q < 3 * n_M; q += kStepThreads) s_acc[q] = 0;
    __syncthreads();
    const int i = s_row;
    const int chunk = item - __ldg(a.IP + i);
    load_row_prefix(a.hist_in, i, n_M, s_n, s_pre, s_wsum);
    __syncthreads();

    const int Ti = s_pre[n_M];
    const uint32_t base = (uint32_t)__ldg(a.R + i);
    int orow[3];
    unsigned long long thr[3];
    double gam[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int c = i - 1 + d;
      orow[d] = (c >= 0 && c < a.n_x) ? __ldg(a.row_map + c) : -1;
      thr[d] = orow[d] >= 0 ? __ldg(a.gthr + orow[d]) : 0ull;
      gam[d] = orow[d] >= 0 ? __ldg(a.gamma + orow[d]) : 0.0;
    }

    const int lo = chunk * kChunk + tid * kPerThread;
    const int hi = min(lo + kPerThread, Ti);
    if (lo < hi) {
      int k = bucket_of(s_pre, n_M, lo);
      int end_k = s_pre[k + 1];
      int sgn = s_n[k] > 0 ? 1 : -1;
      float Dk = s_D[k];
      int cnt[3] = {0, 0, 0};
      for (int lid = lo; lid < hi; ++lid) {
        if (lid >= end_k) {
#pragma unroll
          for (int d = 0; d < 3; ++d)
            if (cnt[d]) {
              atomicAdd(&s_acc[d * n_M + k], sgn * cnt[d]);
              cnt[d] = 0;
            }
          do { ++k; } while (s_pre[k + 1] <= lid);
          end_k = s_pre[k + 1];
          sgn = s_n[k] > 0 ? 1 : -1;
          Dk = s_D[k];
        }
        const uint32_t id = base + (uint32_t)lid;
        int dc = 0;
        if (Dk != 0.f) {
          const uint4 w = philox4x32_10(make_uint4(id, t - 1u, kPurposeRepos, a.sim), a.k0, a.k1);
          const float f = (float)(w.x >> 8) * 0x1p-24f;
          const float fn = __fadd_rn(f, Dk);
          dc = fn >= 1.f ? 1 : (fn < 0.f ? -1 : 0);
        }
        const int c = i + dc;
        if (c < 0 || c >= a.n_x) {
          ++absorbed;
          abs_signed += sgn;
          continue;
        }
        const int d = dc + 1;
        ++cnt[d];
        if (thr[d]) {
          const uint4 w = philox4x32_10(make_uint4(id, t, kPurposeGen, a.sim), a.k0, a.k1);
          const unsigned long long U = ((unsigned long long)(w.x >> 5) << 26) | (unsigned long long)(w.y >> 6);
          if (U < thr[d]) {
            const unsigned long long U2 = ((unsigned long long)(w.z >> 5) << 26) | (unsigned long long)(w.w >> 6);
            const double target = __dmul_rn((double)U2 * 0x1p-53, gam[d]);
            const int kp = sample_momentum(a, orow[d], target);
            if (kp >= 0) {
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
          }
        }
      }
#pragma unroll
      for (int d = 0; d < 3; ++d)
        if (cnt[d]) atomicAdd(&s_acc[d * n_M + k], sgn * cnt[d]);
    }
    __syncthreads();
    for (int q = tid; q < 3 * n_M; q += kStepThreads) {
      const int v = s_acc[q];
      if (v) {
        const int d = q / n_M, kc = q - d * n_M;
        atomicAdd(a.hist_out + (size_t)(i - 1 + d) * n_M + kc, v);
      }
    }
  }

  // block totals of the counters, one atomic each
  const int lane = tid & 31, wid = tid >> 5;
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

static size_t step_smem(int n_M) { return sizeof(int) * (size_t)(n_M + 1 + n_M + 3 * n_M) + sizeof(float) * n_M; }

static int step_grid(int n_M) {
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
  const int g = per_sm * num_sms();
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
  a.IP = v.IP;
  a.row_map = v.row_map;
  a.cdf = v.cdf;
  a.ld = layout(p).ld;
  a.gamma = v.gamma;
  a.gthr = v.gthr;
  a.D = v.D;
  a.VWh = v.VWh;
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
  k_step<<<step_grid(p.n_M), kStepThreads, step_smem(p.n_M), s>>>(a);
  return cudaGetLastError();
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
    const int lo = chunk * kChunk + tid * kPerThread;
    const int hi = min(lo + kPerThread, Ti);
    if (lo < hi) {
      int k = bucket_of(s_pre, n_M, lo);
      for (int lid = lo; lid < hi; ++lid) {
        while (s_pre[k + 1] <= lid) ++k;
        const uint32_t id = base + (uint32_t)lid;
        const uint4 w = philox4x32_10(make_uint4(id, t, kPurposeRepos, sim), k0, k1);
        cell[id] = i;
        f[id] = (float)(w.x >> 8) * 0x1p-24f;
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
