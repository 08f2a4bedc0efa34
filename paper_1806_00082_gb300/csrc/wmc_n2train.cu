// The trained N = 2 network of Sec. 2.3: Eq. (kernel_ML) with N = 2 (one cosine
// factor), its weights learnt by stochastic gradient descent on a
// mean-squared-error loss against exact kernels, one example per step.
//
// Reduced units (kernels times hbar Q / 2, V in eV):
//   y(i, j) = cos(pi j / Q) sum_{d in D(i)} W[d] (wv1 V(i + d) + wv2 V(i + d + 1))
//                                         sin(2 pi j / Q (wt1 d + wt2 (d + 1))),
// D(i) = {d in [-h, h - 1] : i + d even}: the absolute cell pairs (2q, 2q + 1),
// 2q = i + d, inside the window [i - h, i + h]; W indexed by d + h.  The
// parameters are one vector [W[0 .. Q-1], wv1, wv2, wt1, wt2]; at W = -1,
// wv = (1, 1), wt = (1/2, 1/2) the model is the analytic N = 2 network.
//
// Loss of one example: mean over i in [0, n_x), j in [1, h) of (y - t)^2;
// gradient, with G(i, d) = sum_j dL/dy c_j sin(.), H(i, d) = sum_j dL/dy c_j
// phi_j cos(.), phi_j = 2 pi j / Q, P = wv1 V(i+d) + wv2 V(i+d+1):
//   dW[d] = sum_i P G,  dwv1 = sum W V(i+d) G,  dwv2 = sum W V(i+d+1) G,
//   dwt1 = sum W P H d, dwt2 = sum W P H (d + 1).
//
// k_n2_train: one CTA per training run (runs differ in learning rate; they
// train on the same examples in the same order), the whole SGD loop inside the
// CTA: per step the phase tables (sincospif of the current wt), the residuals
// in shared memory, the gradient reductions in a fixed order (a run is
// deterministic) and the update.  No step waits on another CTA.
// k_n2_eval: the trained model's rows, in 1/s, for given parameters.
#include "wmc_device.cuh"

namespace wmc {

namespace {

constexpr int kN2Threads = 1024;
constexpr float kPiF = 3.14159265358979f;  // pi rounded to FP32
constexpr int kN2Warps = kN2Threads / 32;

// Shared memory of k_n2_train: sin and phi-weighted cos tables [Q][h],
// residuals and the products W P [n_x][h] each, V over [-h, n_x + h], cos(pi j
// / Q) [h], the parameters, the W gradient, reduction scratch.
__host__ __device__ inline size_t n2_smem_floats(int n_x, int Q) {
  const int h = Q / 2;
  return 2 * (size_t)Q * h + 2 * (size_t)n_x * h + (size_t)(n_x + Q + 2) + (size_t)h + (size_t)(Q + 4) +
         (size_t)Q + (size_t)6 * kN2Warps;
}

__device__ __forceinline__ float n2_pot(const float* __restrict__ V, int n_x, int bc, int l) {
  if (l >= 0 && l < n_x) return __ldg(V + l);
  if (!bc) return 0.f;
  return __ldg(V + (l < 0 ? 0 : n_x - 1));
}

// Sum of v over the block in a fixed order (warp shuffles, then warp 0);
// every thread gets the result.
__device__ __forceinline__ float n2_block_sum(float v, float* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  float s = 0.f;
  for (int w = 0; w < kN2Warps; ++w) s += red[w];
  return s;
}

}  // namespace

__global__ __launch_bounds__(kN2Threads) void k_n2_train(int n_x, int Q, int bc, int n_ex, const float* __restrict__ Vs,
                                                          const float* __restrict__ VW, float scale, int epochs,
                                                          const int* __restrict__ order, const float* __restrict__ lr,
                                                          float* __restrict__ params, float* __restrict__ loss_out) {
  extern __shared__ float sm_n2[];
  const int h = Q / 2, run = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  float* sS = sm_n2;                       // [Q][h] sin(2 pi j / Q (wt1 d + wt2 (d + 1)))
  float* sC = sS + (size_t)Q * h;          // [Q][h] phi_j times the cosines
  // residuals times (2 / n_out) cos(pi j / Q), by row parity: [2][h][n_x / 2]
  // (lanes of one offset read consecutive rows of one parity without bank conflicts)
  float* sR = sC + (size_t)Q * h;
  float* sWP = sR + (size_t)n_x * h;       // [h][n_x]: W[d] P(i, d) of the k-th pair of row i
  float* sV = sWP + (size_t)n_x * h;       // V(l) at l + h, l in [-h, n_x + h]
  float* sCJ = sV + (n_x + Q + 2);         // cos(pi j / Q)
  float* sP = sCJ + h;                     // parameters
  float* sGW = sP + (Q + 4);               // dL/dW
  float* red = sGW + Q;                    // [6][warps]
  const float rate = __ldg(lr + run);
  float* prm = params + (size_t)run * (Q + 4);
  for (int q = tid; q < Q + 4; q += kN2Threads) sP[q] = prm[q];
  for (int j = tid; j < h; j += kN2Threads) sCJ[j] = cospif((float)j / (float)Q);
  const float inv_n = 2.f / (float)((long long)n_x * (h - 1));  // d(mean of squares)/dy = inv_n r
  const int half = n_x / 2;
  __syncthreads();
  for (int ep = 0; ep < epochs; ++ep) {
    float ep_loss = 0.f;
    for (int s = 0; s < n_ex; ++s) {
      const int ex = __ldg(order + (size_t)ep * n_ex + s);
      const float* V = Vs + (size_t)ex * n_x;
      const float* T = VW + (size_t)ex * n_x * h;
      const float wv1 = sP[Q], wv2 = sP[Q + 1], wt1 = sP[Q + 2], wt2 = sP[Q + 3];
      // phase tables of the current wt and the example's potential
      for (int q = tid; q < Q * h; q += kN2Threads) {
        const int d = q / h - h, j = q % h;
        float sv, cv;
        sincospif(2.f * (float)j / (float)Q * (wt1 * (float)d + wt2 * (float)(d + 1)), &sv, &cv);
        sS[q] = sv;
        sC[q] = cv * (2.f * (float)j / (float)Q) * kPiF;
      }
      for (int l = tid - h; l <= n_x + h; l += kN2Threads) sV[l + h] = n2_pot(V, n_x, bc, l);
      __syncthreads();
      for (int q = tid; q < n_x * h; q += kN2Threads) {  // W[d] P(i, d), k-th pair of row i
        const int k = q / n_x, i = q % n_x;
        const int d = (((i - h) & 1) == 0 ? -h : -h + 1) + 2 * k;
        sWP[q] = sP[d + h] * fmaf(wv1, sV[i + d + h], wv2 * sV[i + d + 1 + h]);
      }
      __syncthreads();
      // residuals (thread q: column j = q / n_x, row i = q % n_x)
      float part = 0.f;
      for (int q = tid; q < n_x * h; q += kN2Threads) {
        const int j = q / n_x, i = q % n_x;
        float r = 0.f;
        if (j > 0) {
          const int dd0 = ((i - h) & 1) == 0 ? 0 : 1;  // d + h of the first pair
          float acc = 0.f;
          for (int k = 0; k < h; ++k) acc = fmaf(sWP[(size_t)k * n_x + i], sS[(dd0 + 2 * k) * h + j], acc);
          r = fmaf(sCJ[j], acc, -__ldg(T + (size_t)i * h + j) * scale);
        }
        sR[((size_t)(i & 1) * h + j) * half + (i >> 1)] = r * sCJ[j] * inv_n;
        part = fmaf(r, r, part);
      }
      const float loss = n2_block_sum(part, red) * (0.5f * inv_n);
      ep_loss += loss;
      // gradients: warp w takes the offsets d = w - h, w + warps - h, ...; its
      // lanes take the rows i = (d & 1) + 2 m of each
      float gv1 = 0.f, gv2 = 0.f, gt1 = 0.f, gt2 = 0.f;
      for (int dd = wid; dd < Q; dd += kN2Warps) {
        const int d = dd - h;
        const float Wd = sP[dd];
        float gw = 0.f;
        const float* rp = sR + (size_t)(d & 1) * h * half;
        for (int m = lane; m < half; m += 32) {
          const int i = (d & 1) + 2 * m;
          float G = 0.f, H = 0.f;
          for (int j = 1; j < h; ++j) {
            const float rc = rp[(size_t)j * half + m];
            G = fmaf(rc, sS[dd * h + j], G);
            H = fmaf(rc, sC[dd * h + j], H);
          }
          const float Va = sV[i + d + h], Vb = sV[i + d + 1 + h];
          const float P = fmaf(wv1, Va, wv2 * Vb);
          gw = fmaf(P, G, gw);
          gv1 = fmaf(Wd * Va, G, gv1);
          gv2 = fmaf(Wd * Vb, G, gv2);
          gt1 = fmaf(Wd * P * H, (float)d, gt1);
          gt2 = fmaf(Wd * P * H, (float)(d + 1), gt2);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) gw += __shfl_down_sync(0xffffffffu, gw, off);
        if (lane == 0) sGW[dd] = gw;
      }
      const float Gv1 = n2_block_sum(gv1, red), Gv2 = n2_block_sum(gv2, red + kN2Warps);
      const float Gt1 = n2_block_sum(gt1, red + 2 * kN2Warps), Gt2 = n2_block_sum(gt2, red + 3 * kN2Warps);
      // update (every thread has read the parameters it needs for this step)
      for (int dd = tid; dd < Q; dd += kN2Threads) sP[dd] = fmaf(-rate, sGW[dd], sP[dd]);
      if (tid == 0) {
        sP[Q] = fmaf(-rate, Gv1, wv1);
        sP[Q + 1] = fmaf(-rate, Gv2, wv2);
        sP[Q + 2] = fmaf(-rate, Gt1, wt1);
        sP[Q + 3] = fmaf(-rate, Gt2, wt2);
      }
      __syncthreads();
    }
    if (tid == 0 && loss_out) loss_out[(size_t)run * epochs + ep] = ep_loss / (float)n_ex;
  }
  for (int q = tid; q < Q + 4; q += kN2Threads) prm[q] = sP[q];
}

// Rows of the trained model in 1/s: row = potential b, cell i (b n_x + i),
// columns j = 0 .. h - 1; one block per row group stages the phase tables.
__global__ __launch_bounds__(256) void k_n2_eval(int n_x, int Q, int bc, long long rows, const float* __restrict__ V,
                                                 const float* __restrict__ prm, float inv_scale,
                                                 float* __restrict__ out) {
  extern __shared__ float sm_e[];
  const int h = Q / 2;
  float* sS = sm_e;            // [Q][h]
  float* sP = sS + (size_t)Q * h;
  for (int q = threadIdx.x; q < Q + 4; q += blockDim.x) sP[q] = __ldg(prm + q);
  __syncthreads();
  const float wv1 = sP[Q], wv2 = sP[Q + 1], wt1 = sP[Q + 2], wt2 = sP[Q + 3];
  for (int q = threadIdx.x; q < Q * h; q += blockDim.x) {
    const int d = q / h - h, j = q % h;
    sS[q] = sinpif(2.f * (float)j / (float)Q * (wt1 * (float)d + wt2 * (float)(d + 1)));
  }
  __syncthreads();
  const long long total = rows * h;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const long long row = q / h;
    const int j = (int)(q % h), i = (int)(row % n_x);
    const float* Vb = V + (size_t)(row / n_x) * n_x;
    float acc = 0.f;
    const int d0 = ((i - h) & 1) == 0 ? -h : -h + 1;
    for (int k = 0; k < h; ++k) {
      const int d = d0 + 2 * k;
      const float P = fmaf(wv1, n2_pot(Vb, n_x, bc, i + d), wv2 * n2_pot(Vb, n_x, bc, i + d + 1));
      acc = fmaf(sP[d + h] * P, sS[(d + h) * h + j], acc);
    }
    out[q] = j ? cospif((float)j / (float)Q) * acc * inv_scale : 0.f;
  }
}

}  // namespace wmc

using namespace wmc;

extern "C" {

wmc_status wmc_n2_train(const wmc_params* p, int32_t n_examples, const float* V, const float* VW, int32_t epochs,
                        const int32_t* order, int32_t n_runs, const float* lr, float* params, float* loss,
                        wmc_stream_t stream) {
  if (!params_ok(p) || n_examples <= 0 || epochs < 0 || n_runs < 0 || !V || !VW || !order || !lr || !params)
    return WMC_ERR_ARG;
  if (p->n_x % 2 != 0) return WMC_ERR_ARG;
  const size_t sm = sizeof(float) * n2_smem_floats(p->n_x, p->Q);
  if (sm > 200 * 1024) return WMC_ERR_UNSUPPORTED;
  if (n_runs == 0 || epochs == 0) return WMC_OK;
  if (sm > 48 * 1024 &&
      raise_smem_limit(reinterpret_cast<const void*>(k_n2_train), sm) != cudaSuccess)
    return WMC_ERR_CUDA;
  const float scale = (float)(kHbarEVs * (double)p->Q / 2.0);
  k_n2_train<<<n_runs, kN2Threads, sm, (cudaStream_t)stream>>>(p->n_x, p->Q, p->bc_potential, n_examples, V, VW,
                                                               scale, epochs, order, lr, params, loss);
  return cudaGetLastError() == cudaSuccess ? WMC_OK : WMC_ERR_CUDA;
}

wmc_status wmc_n2_eval(const wmc_params* p, const float* params, const float* V, int32_t n_pot, float* VWh,
                       wmc_stream_t stream) {
  if (!params_ok(p) || !params || !V || !VWh || n_pot < 0) return WMC_ERR_ARG;
  const long long rows = (long long)n_pot * p->n_x;
  if (rows == 0) return WMC_OK;
  const int h = p->Q / 2;
  const size_t sm = sizeof(float) * ((size_t)p->Q * h + (size_t)(p->Q + 4));
  if (sm > 200 * 1024) return WMC_ERR_UNSUPPORTED;
  if (sm > 48 * 1024 &&
      raise_smem_limit(reinterpret_cast<const void*>(k_n2_eval), sm) != cudaSuccess)
    return WMC_ERR_CUDA;
  long long blocks = (rows * h + 255) / 256;
  if (blocks > 8LL * num_sms()) blocks = 8LL * num_sms();
  const float inv_scale = (float)(2.0 / (kHbarEVs * (double)p->Q));
  k_n2_eval<<<(unsigned)blocks, 256, sm, (cudaStream_t)stream>>>(p->n_x, p->Q, p->bc_potential, rows, V, params,
                                                                 inv_scale, VWh);
  return cudaGetLastError() == cudaSuccess ? WMC_OK : WMC_ERR_CUDA;
}

}  // extern "C"
