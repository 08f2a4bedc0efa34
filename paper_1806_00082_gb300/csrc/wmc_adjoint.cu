// Differentiation form: the adjoint of the kernel rows and of gamma with
// respect to the potential, and of the potential with respect to the
// parameters of a smooth multi-barrier model.
//
// Potential (lengths in nm, energies in eV, x_l = (l + 1/2) dx):
//   V(x) = sum_b h_b T(x; c_b - w_b/2, c_b + w_b/2) + sum_s o_s T(x; s L/ns, (s+1) L/ns),
//   T(x; a, b) = (tanh((x - a)/eps) - tanh((x - b)/eps)) / 2,
// parameters per potential theta = [h_0..h_{nb-1}, w_0.., c_0.., o_0..o_{ns-1}].
//
// Kernel rows (Eq. wigner-1d-discrete, folded): VWh[i][r] = c sum_{m=1}^{h-1} S[m][r] (V(i+m) - V(i-m)),
// gamma[i] = sum over the momentum grid of V_W^+ (Eq. momentum_integral), where
// the column r of a half-period row appears cnt_pos(r) times with sign + and
// cnt_neg(r) times with sign - on the grid; so
//   d gamma / d VWh[i][r] = cnt_pos(r) [VWh > 0] - cnt_neg(r) [VWh < 0].
// Backward, for upstream gVW[i][r] and g_gamma[i]:
//   Gbar[i][r] = gVW[i][r] + g_gamma[i] d gamma / d VWh[i][r],
//   Abar[i][m] = c sum_r Gbar[i][r] S[m][r]                (a contraction, on the tensor cores),
//   Vbar[l]    = sum_m Abar[l-m][m] - Abar[l+m][m]          (V = 0 outside the domain),
//   theta_bar  = sum_l Vbar[l] dV(x_l)/d theta.
#include "wmc_device.cuh"

namespace wmc {

namespace {

// 1 - |tanh u| = 2 / (e^{2|u|} + 1), accurate where tanh saturates.
__device__ __forceinline__ float tanh_tail(float u) { return 2.f / (expf(2.f * fabsf(u)) + 1.f); }

// sech^2 u = 4 e^{-2|u|} / (1 + e^{-2|u|})^2 (no cancellation for large |u|).
__device__ __forceinline__ float sech2(float u) {
  const float e = expf(-2.f * fabsf(u));
  const float d = 1.f + e;
  return 4.f * e / (d * d);
}

// tanh(up) - tanh(um), in tail form when both have the same sign.
__device__ __forceinline__ float tanh_diff(float up, float um) {
  if (up > 0.f && um > 0.f) return tanh_tail(um) - tanh_tail(up);
  if (up < 0.f && um < 0.f) return tanh_tail(up) - tanh_tail(um);
  return tanhf(up) - tanhf(um);
}

__device__ __forceinline__ float window(float x, float a, float b, float inv_eps) {
  return 0.5f * tanh_diff((x - a) * inv_eps, (x - b) * inv_eps);
}

}  // namespace

// ---------------------------------------------------------------- potential
__global__ void k_potential_tanh(const float* __restrict__ theta, int n_pot, int nb, int ns, int n_x, float dx,
                                 float eps, float* __restrict__ V) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= (long long)n_pot * n_x) return;
  const int b = (int)(q / n_x), l = (int)(q % n_x);
  const float* th = theta + (size_t)b * (3 * nb + ns);
  const float x = ((float)l + 0.5f) * dx, inv = 1.f / eps, L = (float)n_x * dx;
  float v = 0.f;
  for (int k = 0; k < nb; ++k) {
    // (x - c) first: exact near the barrier, so the edge is not rounded at |x|
    const float hk = th[k], wk = th[nb + k], xc = x - th[2 * nb + k];
    v += hk * (0.5f * tanh_diff((xc + 0.5f * wk) * inv, (xc - 0.5f * wk) * inv));
  }
  for (int s = 0; s < ns; ++s) v += th[3 * nb + s] * window(x, L * s / ns, L * (s + 1) / ns, inv);
  V[q] = v;
}

// One block per (potential, parameter): each thread keeps a compensated FP32
// sum over a stride of the cells; the block then combines the (sum, error)
// pairs in a fixed tree order, so the result is deterministic.
constexpr int kVjpThreads = 256;

__device__ __forceinline__ void pair_add(float& s, float& e, float s2, float e2) {
  two_sum_acc(s, e, s2);
  e = __fadd_rn(e, e2);
}

__global__ __launch_bounds__(kVjpThreads) void k_potential_tanh_vjp(const float* __restrict__ theta, int n_pot, int nb,
                                                                    int ns, int n_x, float dx, float eps,
                                                                    const float* __restrict__ Vbar,
                                                                    float* __restrict__ theta_bar) {
  __shared__ float red_s[kVjpThreads / 32], red_e[kVjpThreads / 32];
  const int P = 3 * nb + ns;
  const int q = blockIdx.x;
  if (q >= n_pot * P) return;
  const int b = q / P, j = q % P;
  const float* th = theta + (size_t)b * P;
  const float* vb = Vbar + (size_t)b * n_x;
  const float inv = 1.f / eps, L = (float)n_x * dx;
  float s = 0.f, e = 0.f;
  if (j < 3 * nb) {
    const int k = j % nb;
    const float hk = th[k], wk = th[nb + k], ck = th[2 * nb + k];
    for (int l = threadIdx.x; l < n_x; l += kVjpThreads) {
      const float x = ((float)l + 0.5f) * dx;
      const float up = (x - ck + 0.5f * wk) * inv, um = (x - ck - 0.5f * wk) * inv;
      float d;
      if (j < nb) d = 0.5f * tanh_diff(up, um);                           // d/d h_k
      else if (j < 2 * nb) d = hk * (sech2(up) + sech2(um)) * 0.25f * inv;  // d/d w_k
      else d = hk * (sech2(um) - sech2(up)) * 0.5f * inv;                  // d/d c_k
      two_sum_acc(s, e, vb[l] * d);
    }
  } else {
    const int sidx = j - 3 * nb;
    const float a = L * sidx / ns, bb = L * (sidx + 1) / ns;
    for (int l = threadIdx.x; l < n_x; l += kVjpThreads) {
      const float x = ((float)l + 0.5f) * dx;
      two_sum_acc(s, e, vb[l] * window(x, a, bb, inv));  // d/d o_s
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float s2 = __shfl_down_sync(0xffffffffu, s, off), e2 = __shfl_down_sync(0xffffffffu, e, off);
    pair_add(s, e, s2, e2);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red_s[warp] = s, red_e[warp] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    float ts = red_s[0], te = red_e[0];
    for (int w = 1; w < kVjpThreads / 32; ++w) pair_add(ts, te, red_s[w], red_e[w]);
    theta_bar[q] = ts + te;
  }
}

// ---------------------------------------------------------------- Vbar
// Vbar[b][l] = sum_{m=1}^{h-1} Abar[b][l-m][m-1] - Abar[b][l+m][m-1], rows of
// potential b at b n_x .. b n_x + n_x - 1, V = 0 outside the domain.  A block
// computes kVbarTile consecutive cells of one potential: the Abar rows they
// draw on, [l0 - h + 1, l0 + kVbarTile + h - 1), pass through shared memory in
// coalesced chunks of kVbarChunk rows, and thread l adds A[j][l - j - 1] and
// subtracts A[j][j - l - 1] from each staged row j (compensated FP32, rows in
// increasing order).
constexpr int kVbarTile = 256, kVbarChunk = 32;

__global__ __launch_bounds__(kVbarTile) void k_adj_vbar(int Q, int n_x, int n_pot, const float* __restrict__ Abar,
                                                        float* __restrict__ Vbar) {
  extern __shared__ float s_A[];  // kVbarChunk x h
  const int h = Q / 2;
  const int tiles = (n_x + kVbarTile - 1) / kVbarTile;
  const int b = blockIdx.x / tiles, l0 = (blockIdx.x % tiles) * kVbarTile;
  if (b >= n_pot) return;
  const int l = l0 + threadIdx.x;
  const float* Ab = Abar + (size_t)b * n_x * h;
  const int j_lo = max(0, l0 - (h - 1)), j_hi = min(n_x, l0 + kVbarTile + h - 1);
  float s = 0.f, e = 0.f;
  for (int j0 = j_lo; j0 < j_hi; j0 += kVbarChunk) {
    const int nj = min(kVbarChunk, j_hi - j0);
    __syncthreads();
    for (int q = threadIdx.x; q < nj * h; q += kVbarTile) s_A[q] = __ldg(Ab + (size_t)j0 * h + q);
    __syncthreads();
    for (int jj = 0; jj < nj; ++jj) {
      const int j = j0 + jj;
      const int mp = l - j, mn = j - l;  // row j feeds Vbar[j + m] with +, Vbar[j - m] with -
      if (mp >= 1 && mp <= h - 1) two_sum_acc(s, e, s_A[jj * h + mp - 1]);
      else if (mn >= 1 && mn <= h - 1) two_sum_acc(s, e, -s_A[jj * h + mn - 1]);
    }
  }
  if (l < n_x) Vbar[(size_t)b * n_x + l] = s + e;
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_potential_tanh(const float* theta, int n_pot, int nb, int ns, int n_x, float dx, float eps,
                                  float* V, cudaStream_t s) {
  const long long n = (long long)n_pot * n_x;
  if (n <= 0) return cudaSuccess;
  k_potential_tanh<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(theta, n_pot, nb, ns, n_x, dx, eps, V);
  return cudaGetLastError();
}

cudaError_t launch_potential_tanh_vjp(const float* theta, int n_pot, int nb, int ns, int n_x, float dx, float eps,
                                      const float* Vbar, float* theta_bar, cudaStream_t s) {
  const int n = n_pot * (3 * nb + ns);
  if (n <= 0) return cudaSuccess;
  k_potential_tanh_vjp<<<n, kVjpThreads, 0, s>>>(theta, n_pot, nb, ns, n_x, dx, eps, Vbar, theta_bar);
  return cudaGetLastError();
}

cudaError_t launch_kernel_vjp(const wmc_params& p, int n_pot, const float* VWh, const float* gVW,
                              const float* g_gamma, const void* tc_images, unsigned int* flags, float* Abar,
                              float* Vbar, cudaStream_t s) {
  const int h = p.Q / 2, rows = n_pot * p.n_x;
  if (rows <= 0) return cudaSuccess;
  // Abar = c Gbar S^T: the contraction on the tensor cores (3xTF32 split)
  cudaError_t e = launch_adjoint_abar_tc(p, rows, VWh, gVW, g_gamma, tc_images, Abar, flags, s);
  if (e != cudaSuccess) return e;
  const int tiles = (p.n_x + kVbarTile - 1) / kVbarTile;
  const size_t vsm = sizeof(float) * (size_t)kVbarChunk * h;
  if (vsm > 48 * 1024) raise_smem_limit(reinterpret_cast<const void*>(k_adj_vbar), vsm);
  k_adj_vbar<<<(unsigned)((long long)tiles * n_pot), kVbarTile, vsm, s>>>(p.Q, p.n_x, n_pot, Abar, Vbar);
  return cudaGetLastError();
}

}  // namespace wmc

using namespace wmc;

extern "C" {

wmc_status wmc_potential_tanh(const wmc_params* p, const float* theta, int32_t n_pot, int32_t n_barriers,
                              int32_t n_segments, float eps_nm, float* V, wmc_stream_t stream) {
  if (!params_ok(p) || !theta || !V || n_pot < 0 || n_barriers < 0 || n_segments < 0 || !(eps_nm > 0.f))
    return WMC_ERR_ARG;
  return launch_potential_tanh(theta, n_pot, n_barriers, n_segments, p->n_x, (float)(p->dx_m * 1e9), eps_nm, V,
                               (cudaStream_t)stream) == cudaSuccess
             ? WMC_OK
             : WMC_ERR_CUDA;
}

wmc_status wmc_potential_tanh_vjp(const wmc_params* p, const float* theta, int32_t n_pot, int32_t n_barriers,
                                  int32_t n_segments, float eps_nm, const float* Vbar, float* theta_bar,
                                  wmc_stream_t stream) {
  if (!params_ok(p) || !theta || !Vbar || !theta_bar || n_pot < 0 || n_barriers < 0 || n_segments < 0 ||
      !(eps_nm > 0.f))
    return WMC_ERR_ARG;
  return launch_potential_tanh_vjp(theta, n_pot, n_barriers, n_segments, p->n_x, (float)(p->dx_m * 1e9), eps_nm,
                                   Vbar, theta_bar, (cudaStream_t)stream) == cudaSuccess
             ? WMC_OK
             : WMC_ERR_CUDA;
}

wmc_status wmc_kernel_eval_rows(const wmc_params* p, const float* V, int32_t n_pot, wmc_precision prec, float* VWh,
                                void* ws, wmc_stream_t stream) {
  NvtxRange nvtx("wmc_kernel_eval_rows");
  if (!params_ok(p) || !V || !VWh || !ws || n_pot < 0) return WMC_ERR_ARG;
  if (prec != WMC_FP32 && prec != WMC_BF16 && prec != WMC_FP16 && prec != WMC_FP16_SPLIT && prec != WMC_TF32X3 &&
      prec != WMC_FP32_SIMT)
    return WMC_ERR_UNSUPPORTED;
  const long long rows = (long long)n_pot * p->n_x;
  if (rows == 0) return WMC_OK;
  if (rows > 0x7fffffffll) return WMC_ERR_ARG;
  const View v = view(*p, ws);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  prec = (wmc_precision)resolve_precision(*p, (int)prec, 1, rows);
  if (prec != WMC_FP32)
    e = launch_kernel_eval_tc(*p, (int)prec, V, nullptr, nullptr, (int)rows, (int)rows, v.tc, VWh, &v.hdr->flags, s);
  else if (small_window(*p))
    e = launch_kernel_rows_small(*p, V, nullptr, nullptr, (int)rows, (int)rows, v.B, VWh, nullptr, nullptr, nullptr,
                                 nullptr, nullptr, nullptr, s);
  else
    e = launch_kernel_eval(*p, V, nullptr, nullptr, (int)rows, (int)rows, v.B, VWh, s);
  return e == cudaSuccess ? WMC_OK : WMC_ERR_CUDA;
}

wmc_status wmc_kernel_vjp(const wmc_params* p, const float* VWh, const float* gVW, const float* g_gamma,
                          int32_t n_pot, float* Abar, float* Vbar, void* ws, wmc_stream_t stream) {
  NvtxRange nvtx("wmc_kernel_vjp");
  if (!params_ok(p) || !VWh || !Abar || !Vbar || !ws || n_pot < 0 || (!gVW && !g_gamma)) return WMC_ERR_ARG;
  if (p->bc_potential != 0 || p->Q / 2 > kAdjMaxH) return WMC_ERR_UNSUPPORTED;
  const View v = view(*p, ws);
  return launch_kernel_vjp(*p, n_pot, VWh, gVW, g_gamma, v.tc, &v.hdr->flags, Abar, Vbar, (cudaStream_t)stream) ==
                 cudaSuccess
             ? WMC_OK
             : WMC_ERR_CUDA;
}

}  // extern "C"
