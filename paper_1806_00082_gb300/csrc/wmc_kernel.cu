// Wigner kernel on occupied cells -- Eq. (wigner-1d-discrete) evaluated as the
// N = 1 analytic network of Sec. 2.2 -- and the gamma / momentum-CDF epilogue
// of Eq. (momentum_integral).
//
// Contraction (folded over the odd symmetry of the window sum):
//   VWh[row][r] = c * sum_{m=1}^{h-1} A[row][m] * S[m][r],  c = -2 / (hbar Q)
//   A[row][m]   = V(i+m) - V(i-m),  i = occ[row]   (built on the fly from V)
//   S[m][r]     = sin(2 pi (m r mod Q) / Q)          (precomputed matrix B)
#include <math.h>

#include "wmc_internal.cuh"

namespace wmc {

__device__ __forceinline__ float pot(const float* __restrict__ V, int n_x, int bc, long long l) {
  if (l >= 0 && l < n_x) return __ldg(V + l);
  if (!bc) return 0.f;
  return __ldg(V + (l < 0 ? 0 : n_x - 1));
}

// Error-free transformation of a + b (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum_acc(float& s, float& e, float p) {
  const float sn = __fadd_rn(s, p);
  const float bp = __fsub_rn(sn, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(sn, bp)), __fsub_rn(p, bp));
  s = sn;
  e = __fadd_rn(e, err);
}

// ---------------------------------------------------------------- FP32 SIMT contraction
// Tile BM x BN outputs per block of 256 threads (4 x 4 per thread), K chunks of
// BK.  Each K chunk is accumulated by FMA into a fresh partial, which is then
// added to the running sum with TwoSum: the accumulation error stays at the
// level of one 32-term chunk instead of growing with the window length.
constexpr int BM = 64, BN = 64, BK = 32;

__global__ __launch_bounds__(256) void k_kernel_eval_fp32(const float* __restrict__ V, int n_x, int bc, int Q,
                                                          const int* __restrict__ occ,
                                                          const int* __restrict__ n_occ_dev, int n_occ_host,
                                                          const float* __restrict__ B, int Kp, int Np, float c,
                                                          float* __restrict__ VWh) {
  __shared__ __align__(16) float As[BK][BM];
  __shared__ __align__(16) float Bs[BK][BN];
  const int n_rows = n_occ_dev ? *n_occ_dev : n_occ_host;
  const int row0 = blockIdx.x * BM, col0 = blockIdx.y * BN;
  const int h = Q / 2;
  if (row0 >= n_rows || col0 >= h) return;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;

  // the A rows this thread builds: r = tid & 63, kk = (tid >> 6) + 4 q
  const int ar = tid & 63;
  const int a_row = row0 + ar;
  const int a_cell = a_row < n_rows ? __ldg(occ + a_row) : 0;

  float s[4][4], e[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) s[a][b] = e[a][b] = 0.f;

  for (int k0 = 0; k0 < Kp; k0 += BK) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int kk = (tid >> 6) + 4 * q;
      const int m = k0 + kk + 1;
      float v = 0.f;
      if (m <= h - 1) v = __fsub_rn(pot(V, n_x, bc, (long long)a_cell + m), pot(V, n_x, bc, (long long)a_cell - m));
      As[kk][ar] = v;
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int idx = tid + 256 * q;
      const int kk = idx >> 4, c4 = (idx & 15) * 4;
      *reinterpret_cast<float4*>(&Bs[kk][c4]) =
          __ldg(reinterpret_cast<const float4*>(B + (size_t)(k0 + kk) * Np + col0 + c4));
    }
    __syncthreads();
    float p[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) p[a][b] = 0.f;
#pragma unroll 8
    for (int kk = 0; kk < BK; ++kk) {
      const float4 av = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 bv = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float ar4[4] = {av.x, av.y, av.z, av.w};
      const float br4[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) p[a][b] = fmaf(ar4[a], br4[b], p[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) two_sum_acc(s[a][b], e[a][b], p[a][b]);
    __syncthreads();
  }

#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int row = row0 + ty * 4 + a;
    if (row >= n_rows) continue;
    float* out = VWh + (size_t)row * h;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int col = col0 + tx * 4 + b;
      if (col < h) out[col] = __fmul_rn(c, __fadd_rn(s[a][b], e[a][b]));
    }
  }
}

cudaError_t launch_kernel_eval(const wmc_params& p, const float* V, const int* occ, const int* n_occ_dev,
                               int n_occ_host, int max_rows, const float* B, float* VWh, cudaStream_t s) {
  if (max_rows <= 0) return cudaSuccess;
  const Layout L = layout(p);
  const float c = (float)(-2.0 / (kHbarEVs * (double)p.Q));
  dim3 grid((max_rows + BM - 1) / BM, (L.h + BN - 1) / BN);
  k_kernel_eval_fp32<<<grid, 256, 0, s>>>(V, p.n_x, p.bc_potential, p.Q, occ, n_occ_dev, n_occ_host, B, L.Kp, L.Np,
                                          c, VWh);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- caller table
__global__ void k_gather_table(const float* __restrict__ table, int h, const int* __restrict__ occ,
                               const int* __restrict__ n_occ_dev, float* __restrict__ VWh) {
  const int n_rows = *n_occ_dev;
  for (int row = blockIdx.x; row < n_rows; row += gridDim.x) {
    const float* src = table + (size_t)__ldg(occ + row) * h;
    float* dst = VWh + (size_t)row * h;
    for (int r = threadIdx.x; r < h; r += blockDim.x) dst[r] = __ldg(src + r);
  }
}

cudaError_t launch_gather_table(const wmc_params& p, const float* table, const int* occ, const int* n_occ_dev,
                                int max_rows, float* VWh, cudaStream_t s) {
  if (max_rows <= 0) return cudaSuccess;
  const int blocks = max_rows < 4 * 152 ? max_rows : 4 * 152;
  k_gather_table<<<blocks, 128, 0, s>>>(table, p.Q / 2, occ, n_occ_dev, VWh);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- gamma and CDF
// gamma and the momentum CDF of one kernel row per warp.  The positive parts
// x_k = max(V_W(k), 0) are quantised relative to the row maximum,
//   e = floor(log2 max x),  s = 61 - ceil(log2 n_M) - e,
//   q_k = x_k 2^s rounded to the nearest integer, ties to even,
// so that the CDF C[k] = sum_{k' <= k} q_k' is an exact int64 running sum (any
// summation order gives the same bits, so a warp scan computes it) and
// gamma = fl64(C[n_M-1] 2^-s).  gthr[row] = ceil(fl64(gamma dt) 2^32): for a
// 32-bit word w, w < gthr  <=>  w 2^-32 < gamma dt.

// x 2^s rounded to the nearest integer (ties to even), from the bits of x >= 0.
__device__ __forceinline__ long long quantise(float x, int s) {
  const uint32_t b = __float_as_uint(x);
  if (b == 0u) return 0;
  const uint32_t E = b >> 23;
  uint32_t m = b & 0x7fffffu;
  int ex = -149;                 // value = m 2^ex
  if (E) {
    m |= 0x800000u;
    ex = (int)E - 150;
  }
  const int sh = ex + s;
  if (sh >= 0) return (long long)((unsigned long long)m << sh);
  const int r = -sh;
  if (r > 25) return 0;          // m < 2^24: below half a unit
  const uint32_t q = m >> r;
  const uint32_t rem = m & ((1u << r) - 1u), half = 1u << (r - 1);
  return (long long)(q + ((rem > half || (rem == half && (q & 1u))) ? 1u : 0u));
}

__device__ __forceinline__ int floor_log2_pos(float x) {  // x > 0
  const uint32_t b = __float_as_uint(x);
  const uint32_t E = b >> 23;
  if (E) return (int)E - 127;
  return (31 - __clz(b & 0x7fffffu)) - 149;
}

__device__ __forceinline__ float positive_part(const float* __restrict__ v, int Q, int r) {
  const int h = Q / 2;
  float x = 0.f;
  if (r != 0 && r != h) x = r < h ? __ldg(v + r) : -__ldg(v + (Q - r));
  return x > 0.f ? x : 0.f;
}

constexpr int kCdfWarps = 8;

__global__ __launch_bounds__(kCdfWarps * 32) void k_cdf(int n_M, int Q, int log2_nM, const float* __restrict__ VWh,
                                                       const int* __restrict__ n_rows_dev, int n_rows_host,
                                                       long long* __restrict__ cdf, long long ldk, long long ldr,
                                                       double* __restrict__ gamma, int* __restrict__ scale,
                                                       unsigned long long* __restrict__ gthr,
                                                       const int* __restrict__ occ,
                                                       unsigned long long* __restrict__ thr_cell,
                                                       unsigned int* __restrict__ flags, double dt) {
  const int n_rows = n_rows_dev ? *n_rows_dev : n_rows_host;
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * kCdfWarps + (threadIdx.x >> 5);
  if (row >= n_rows) return;
  const int h = Q / 2;
  const float* v = VWh + (size_t)row * h;
  const int r0 = ((-(n_M / 2)) % Q + Q) % Q;   // r of column k = 0
  // row maximum of the positive parts (non-negative floats order as their bits)
  uint32_t mx = 0u;
  for (int k = lane; k < n_M; k += 32) mx = max(mx, __float_as_uint(positive_part(v, Q, (r0 + k) % Q)));
  mx = __reduce_max_sync(0xffffffffu, mx);
  long long* out = cdf ? cdf + row * ldr : nullptr;
  if (mx == 0u) {
    if (out)
      for (int k = lane; k < n_M; k += 32) out[k * ldk] = 0;
    if (lane == 0) {
      gamma[row] = 0.0;
      if (scale) scale[row] = 0;
      if (gthr) gthr[row] = 0ull;
      if (thr_cell) thr_cell[__ldg(occ + row)] = 0ull;
    }
    return;
  }
  const int s = 61 - log2_nM - floor_log2_pos(__uint_as_float(mx));
  long long carry = 0;
  for (int k0 = 0; k0 < n_M; k0 += 32) {
    const int k = k0 + lane;
    long long q = k < n_M ? quantise(positive_part(v, Q, (r0 + k) % Q), s) : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const long long u = __shfl_up_sync(0xffffffffu, q, off);
      if (lane >= off) q += u;
    }
    q += carry;
    if (out && k < n_M) out[k * ldk] = q;
    carry = __shfl_sync(0xffffffffu, q, 31);
  }
  if (lane == 0) {
    const double g = ldexp((double)carry, -s);
    gamma[row] = g;
    if (scale) scale[row] = s;
    if (gthr) {
      const double gd = __dmul_rn(g, dt);
      unsigned long long thr;
      if (gd >= 1.0) {
        atomicOr(flags, WMC_FLAG_RATE);
        thr = 1ull << 32;
      } else {
        thr = (unsigned long long)ceil(gd * 4294967296.0);
      }
      gthr[row] = thr;
      if (thr_cell) thr_cell[__ldg(occ + row)] = thr;
    }
  }
}

static int ceil_log2(int n) {
  int L = 0;
  while ((1 << L) < n) ++L;
  return L;
}

cudaError_t launch_cdf(const wmc_params& p, const float* VWh, const int* n_rows_dev, int n_rows_host, int max_rows,
                       long long* cdf, long long ldk, long long ldr, double* gamma, int* scale,
                       unsigned long long* gthr, const int* occ, unsigned long long* thr_cell, unsigned int* flags,
                       cudaStream_t s) {
  if (max_rows <= 0) return cudaSuccess;
  k_cdf<<<(max_rows + kCdfWarps - 1) / kCdfWarps, kCdfWarps * 32, 0, s>>>(
      p.n_M, p.Q, ceil_log2(p.n_M), VWh, n_rows_dev, n_rows_host, cdf, ldk, ldr, gamma, scale, gthr, occ, thr_cell,
      flags, p.dt_s);
  return cudaGetLastError();
}

}  // namespace wmc
