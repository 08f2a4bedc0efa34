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
//   Abar[i][m] = c sum_r Gbar[i][r] S[m][r]                (a contraction),
//   Vbar[l]    = sum_m Abar[l-m][m] - Abar[l+m][m]          (V = 0 outside the domain),
//   theta_bar  = sum_l Vbar[l] dV(x_l)/d theta.
#include "wmc_device.cuh"

namespace wmc {

namespace {

// number of momentum indices M in [-n_M/2, n_M/2) with M = r (mod Q)
__device__ __forceinline__ int grid_count(int r, int Q, int n_M) {
  const int M0 = -(n_M / 2);
  const int M1 = M0 + ((((r - M0) % Q) + Q) % Q);
  return M1 < n_M / 2 ? (n_M / 2 - 1 - M1) / Q + 1 : 0;
}

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

// one thread per (potential, parameter): compensated FP32 sum over the cells
__global__ void k_potential_tanh_vjp(const float* __restrict__ theta, int n_pot, int nb, int ns, int n_x, float dx,
                                     float eps, const float* __restrict__ Vbar, float* __restrict__ theta_bar) {
  const int P = 3 * nb + ns;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_pot * P) return;
  const int b = q / P, j = q % P;
  const float* th = theta + (size_t)b * P;
  const float* vb = Vbar + (size_t)b * n_x;
  const float inv = 1.f / eps, L = (float)n_x * dx;
  float s = 0.f, e = 0.f;
  for (int l = 0; l < n_x; ++l) {
    const float x = ((float)l + 0.5f) * dx;
    float d;
    if (j < 3 * nb) {
      const int k = j % nb;
      const float hk = th[k], wk = th[nb + k], ck = th[2 * nb + k];
      const float up = (x - ck + 0.5f * wk) * inv, um = (x - ck - 0.5f * wk) * inv;
      const float sp = sech2(up), sm = sech2(um);
      if (j < nb) d = 0.5f * tanh_diff(up, um);               // d/d h_k
      else if (j < 2 * nb) d = hk * (sp + sm) * 0.25f * inv;  // d/d w_k
      else d = hk * (sm - sp) * 0.5f * inv;                   // d/d c_k
    } else {
      const int sidx = j - 3 * nb;
      d = window(x, L * sidx / ns, L * (sidx + 1) / ns, inv);  // d/d o_s
    }
    two_sum_acc(s, e, vb[l] * d);
  }
  theta_bar[q] = s + e;
}

// ---------------------------------------------------------------- Abar
// One warp per row: Gbar of the row in shared memory, then lane kk (= m - 1)
// accumulates c sum_r Gbar[r] S[m][r] against the transposed sine matrix
// staged in shared memory (compensated FP32 in chunks of 32 terms).
constexpr int kAdjWarps = 8;

template <int C>
__global__ __launch_bounds__(kAdjWarps * 32) void k_adj_abar(int Q, int n_M, int rows, const float* __restrict__ VWh,
                                                             const float* __restrict__ gVW,
                                                             const float* __restrict__ g_gamma,
                                                             const float* __restrict__ B, int Np, float c,
                                                             float* __restrict__ Abar) {
  extern __shared__ float s_mem[];
  const int h = Q / 2;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* s_Bt = s_mem;                                 // [h][32 C]: s_Bt[r][kk] = S[kk+1][r]
  float* s_g = s_mem + h * 32 * C + wid * 32 * C;     // Gbar of this warp's row
  if ((int)(blockIdx.x * kAdjWarps) >= rows) return;
  for (int q = threadIdx.x; q < h * 32 * C; q += blockDim.x) {
    const int r = q / (32 * C), kk = q % (32 * C);
    s_Bt[q] = kk < h - 1 ? __ldg(B + (size_t)kk * Np + r) : 0.f;
  }
  __syncthreads();
  for (int row = blockIdx.x * kAdjWarps + wid; row < rows; row += gridDim.x * kAdjWarps) {
    const float gg = g_gamma ? __ldg(g_gamma + row) : 0.f;
#pragma unroll
    for (int cc = 0; cc < C; ++cc) {
      const int r = lane + 32 * cc;
      float g = 0.f;
      if (r < h) {
        if (gVW) g = __ldg(gVW + (size_t)row * h + r);
        if (gg != 0.f && r > 0) {
          const float v = __ldg(VWh + (size_t)row * h + r);
          const int dg = v > 0.f ? grid_count(r, Q, n_M) : (v < 0.f ? -grid_count(Q - r, Q, n_M) : 0);
          g = __fadd_rn(g, __fmul_rn(gg, (float)dg));
        }
      }
      s_g[r] = g;
    }
    __syncwarp();
    float sacc[C], eacc[C];
#pragma unroll
    for (int q = 0; q < C; ++q) sacc[q] = eacc[q] = 0.f;
    for (int r0 = 0; r0 < h; r0 += 32) {
      float part[C];
#pragma unroll
      for (int q = 0; q < C; ++q) part[q] = 0.f;
      const int r1 = min(r0 + 32, h);
      for (int r = r0; r < r1; ++r) {
        const float g = s_g[r];
        const float* bt = s_Bt + r * 32 * C;
#pragma unroll
        for (int q = 0; q < C; ++q) part[q] = fmaf(g, bt[lane + 32 * q], part[q]);
      }
#pragma unroll
      for (int q = 0; q < C; ++q) two_sum_acc(sacc[q], eacc[q], part[q]);
    }
#pragma unroll
    for (int q = 0; q < C; ++q) {
      const int kk = lane + 32 * q;
      if (kk < h - 1) Abar[(size_t)row * h + kk] = __fmul_rn(c, __fadd_rn(sacc[q], eacc[q]));
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------- Vbar
// Vbar[b][l] = sum_{m=1}^{h-1} Abar[b][l-m][m-1] - Abar[b][l+m][m-1], rows of
// potential b at b n_x .. b n_x + n_x - 1, V = 0 outside the domain.
__global__ void k_adj_vbar(int Q, int n_x, int n_pot, const float* __restrict__ Abar, float* __restrict__ Vbar) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= (long long)n_pot * n_x) return;
  const int h = Q / 2;
  const int b = (int)(q / n_x), l = (int)(q % n_x);
  const float* Ab = Abar + (size_t)b * n_x * h;
  float s = 0.f, e = 0.f;
  for (int m = 1; m <= h - 1; ++m) {
    float t = 0.f;
    if (l - m >= 0) t = __ldg(Ab + (size_t)(l - m) * h + (m - 1));
    if (l + m < n_x) t = __fsub_rn(t, __ldg(Ab + (size_t)(l + m) * h + (m - 1)));
    two_sum_acc(s, e, t);
  }
  Vbar[q] = s + e;
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
  k_potential_tanh_vjp<<<(n + 127) / 128, 128, 0, s>>>(theta, n_pot, nb, ns, n_x, dx, eps, Vbar, theta_bar);
  return cudaGetLastError();
}

cudaError_t launch_kernel_vjp(const wmc_params& p, int n_pot, const float* VWh, const float* gVW,
                              const float* g_gamma, const float* B, float* Abar, float* Vbar, cudaStream_t s) {
  const Layout L = layout(p);
  const int h = L.h, rows = n_pot * p.n_x;
  if (rows <= 0) return cudaSuccess;
  const float c = (float)(-2.0 / (kHbarEVs * (double)p.Q));
  const int C = h <= 32 ? 1 : (h <= 64 ? 2 : 4);
  const size_t sm = sizeof(float) * ((size_t)h * 32 * C + (size_t)kAdjWarps * 32 * C);
  int blocks = (rows + kAdjWarps - 1) / kAdjWarps;
  if (blocks > 4 * num_sms()) blocks = 4 * num_sms();
#define WMC_LAUNCH_ABAR(CC)                                                                                   \
  do {                                                                                                        \
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_adj_abar<CC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
    k_adj_abar<CC><<<blocks, kAdjWarps * 32, sm, s>>>(p.Q, p.n_M, rows, VWh, gVW, g_gamma, B, L.Np, c, Abar);     \
  } while (0)
  if (C == 1) WMC_LAUNCH_ABAR(1);
  else if (C == 2) WMC_LAUNCH_ABAR(2);
  else WMC_LAUNCH_ABAR(4);
#undef WMC_LAUNCH_ABAR
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long n = (long long)rows;
  k_adj_vbar<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p.Q, p.n_x, n_pot, Abar, Vbar);
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
  if (!params_ok(p) || !V || !VWh || !ws || n_pot < 0) return WMC_ERR_ARG;
  if (prec != WMC_FP32 && prec != WMC_BF16 && prec != WMC_FP16 && prec != WMC_FP16_SPLIT) return WMC_ERR_UNSUPPORTED;
  const long long rows = (long long)n_pot * p->n_x;
  if (rows == 0) return WMC_OK;
  if (rows > 0x7fffffffll) return WMC_ERR_ARG;
  const View v = view(*p, ws);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (prec != WMC_FP32)
    e = launch_kernel_eval_tc(*p, (int)prec, V, nullptr, nullptr, (int)rows, (int)rows, v.tc, VWh, &v.hdr->flags, s);
  else if (small_window(*p))
    e = launch_kernel_rows_small(*p, V, nullptr, nullptr, (int)rows, (int)rows, v.B, VWh, nullptr, nullptr, nullptr,
                                 nullptr, nullptr, s);
  else
    e = launch_kernel_eval(*p, V, nullptr, nullptr, (int)rows, (int)rows, v.B, VWh, s);
  return e == cudaSuccess ? WMC_OK : WMC_ERR_CUDA;
}

wmc_status wmc_kernel_vjp(const wmc_params* p, const float* VWh, const float* gVW, const float* g_gamma,
                          int32_t n_pot, float* Abar, float* Vbar, void* ws, wmc_stream_t stream) {
  if (!params_ok(p) || !VWh || !Abar || !Vbar || !ws || n_pot < 0 || (!gVW && !g_gamma)) return WMC_ERR_ARG;
  if (p->bc_potential != 0 || p->Q / 2 > 128) return WMC_ERR_UNSUPPORTED;
  const View v = view(*p, ws);
  return launch_kernel_vjp(*p, n_pot, VWh, gVW, g_gamma, v.B, Abar, Vbar, (cudaStream_t)stream) == cudaSuccess
             ? WMC_OK
             : WMC_ERR_CUDA;
}

}  // extern "C"
