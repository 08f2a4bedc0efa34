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
// One thread per kernel row: the running FP64 sum of V_W^+ over ascending M
// (the order is part of the result: the pair sampler compares against these
// exact partial sums).  gthr[row] = ceil(gamma dt 2^53), so that for a 53-bit
// integer U, U < gthr  <=>  U 2^-53 < gamma dt.
__global__ void k_cdf(int n_M, int Q, const float* __restrict__ VWh, const int* __restrict__ n_rows_dev,
                      int n_rows_host, double* __restrict__ cdf, long long ldk, long long ldr,
                      double* __restrict__ gamma, unsigned long long* __restrict__ gthr,
                      unsigned int* __restrict__ flags, double dt) {
  const int n_rows = n_rows_dev ? *n_rows_dev : n_rows_host;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n_rows) return;
  const int h = Q / 2;
  const float* v = VWh + (size_t)row * h;
  int r = (-(n_M / 2)) % Q;
  if (r < 0) r += Q;
  double acc = 0.0;
  double* out = cdf ? cdf + row * ldr : nullptr;
  for (int k = 0; k < n_M; ++k) {
    float x = 0.f;
    if (r != 0 && r != h) x = r < h ? __ldg(v + r) : -__ldg(v + (Q - r));
    const double xd = (double)x;
    acc = __dadd_rn(acc, xd > 0.0 ? xd : 0.0);
    if (out) out[k * ldk] = acc;
    if (++r == Q) r = 0;
  }
  gamma[row] = acc;
  if (gthr) {
    const double g = __dmul_rn(acc, dt);
    unsigned long long thr;
    if (g >= 1.0) {
      atomicOr(flags, WMC_FLAG_RATE);
      thr = 1ull << 53;
    } else {
      thr = (unsigned long long)ceil(g * 9007199254740992.0);
    }
    gthr[row] = thr;
  }
}

cudaError_t launch_cdf(const wmc_params& p, const float* VWh, const int* n_rows_dev, int n_rows_host, int max_rows,
                       double* cdf, long long ldk, long long ldr, double* gamma, unsigned long long* gthr,
                       unsigned int* flags, cudaStream_t s) {
  if (max_rows <= 0) return cudaSuccess;
  const int threads = 128;
  k_cdf<<<(max_rows + threads - 1) / threads, threads, 0, s>>>(p.n_M, p.Q, VWh, n_rows_dev, n_rows_host, cdf, ldk,
                                                               ldr, gamma, gthr, flags, p.dt_s);
  return cudaGetLastError();
}

}  // namespace wmc
