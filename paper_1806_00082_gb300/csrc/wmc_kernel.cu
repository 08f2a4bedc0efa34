// Wigner kernel on occupied cells -- Eq. (wigner-1d-discrete) evaluated as the
// N = 1 analytic network of Sec. 2.2 -- and the gamma / momentum-CDF epilogue
// of Eq. (momentum_integral).
//
// Contraction (folded over the odd symmetry of the window sum):
//   VWh[row][r] = c * sum_{m=1}^{h-1} A[row][m] * S[m][r],  c = -2 / (hbar Q)
//   A[row][m]   = V(i+m) - V(i-m),  i = occ[row]   (built on the fly from V)
//   S[m][r]     = sin(2 pi (m r mod Q) / Q)          (precomputed matrix B)
#include <math.h>

#include "wmc_device.cuh"

namespace wmc {

// ---------------------------------------------------------------- FP32 SIMT contraction
// Tile BM x BN outputs per block of 256 threads (4 x 4 per thread), K chunks of
// BK.  Each K chunk is accumulated by FMA into a fresh partial, which is then
// added to the running sum with TwoSum: the accumulation error stays at the
// level of one 32-term chunk instead of growing with the window length.
constexpr int BM = 64, BN = 64, BK = 32;

template <int NET>
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
  // occ == nullptr: implicit rows over consecutive potentials (row r is cell
  // r % n_x of the potential V + (r / n_x) n_x)
  const int a_cell = a_row < n_rows ? (occ ? __ldg(occ + a_row) : a_row % n_x) : 0;
  const float* Va = (occ || a_row >= n_rows) ? V : V + (size_t)(a_row / n_x) * n_x;

  float s[4][4], e[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) s[a][b] = e[a][b] = 0.f;

  for (int k0 = 0; k0 < Kp; k0 += BK) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int kk = (tid >> 6) + 4 * q;
      const float v = a_term<NET>(Va, n_x, bc, h, a_cell, k0 + kk);
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
                               int n_occ_host, int max_rows, const float* B, float* VWh, cudaStream_t s, int net) {
  if (max_rows <= 0) return cudaSuccess;
  const Layout L = layout(p);
  const float c = (float)(-2.0 / (kHbarEVs * (double)p.Q));
  dim3 grid((max_rows + BM - 1) / BM, (L.h + BN - 1) / BN);
  if (net == 2)
    k_kernel_eval_fp32<2><<<grid, 256, 0, s>>>(V, p.n_x, p.bc_potential, p.Q, occ, n_occ_dev, n_occ_host, B, L.Kp2,
                                               L.Np, c, VWh);
  else
    k_kernel_eval_fp32<1><<<grid, 256, 0, s>>>(V, p.n_x, p.bc_potential, p.Q, occ, n_occ_dev, n_occ_host, B, L.Kp,
                                               L.Np, c, VWh);
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

constexpr int kCdfWarps = 8;

__global__ __launch_bounds__(kCdfWarps * 32) void k_cdf(int n_M, int Q, int log2_nM, const float* __restrict__ VWh,
                                                       const int* __restrict__ n_rows_dev, int n_rows_host,
                                                       long long* __restrict__ cdf, double* __restrict__ gamma,
                                                       int* __restrict__ scale, unsigned long long* __restrict__ gthr,
                                                       const int* __restrict__ occ,
                                                       unsigned long long* __restrict__ thr_cell,
                                                       unsigned int* __restrict__ flags, double dt,
                                                       DevHeader* __restrict__ hdr, long long* __restrict__ ccdf) {
  extern __shared__ float s_cdf_rows[];  // one staged row (Q / 2 floats) per warp
  const int n_rows = n_rows_dev ? *n_rows_dev : n_rows_host;
  if (hdr && blockIdx.x == 0 && threadIdx.x == 0) hdr->rows_by_cell = 0u;  // rows follow the occupied list
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * kCdfWarps + (threadIdx.x >> 5);
  if (row >= n_rows) return;
  const int h = Q / 2;
  // the row is staged in shared memory by coalesced loads: the CDF reads it
  // in grid order (a permutation of the folded row), once per pass
  // (padded: element r at r + r / 32, so that the lanes' contiguous column
  // runs fall in distinct banks)
  float* sv = s_cdf_rows + (threadIdx.x >> 5) * (h + h / 32 + 1);
  const float* v = VWh + (size_t)row * h;
  for (int r = lane; r < h; r += 32) sv[r + (r >> 5)] = __ldg(v + r);
  __syncwarp();
  const int r0 = ((-(n_M / 2)) % Q + Q) % Q;   // r of column k = 0
  auto xres = [&](int rr) {
    float x = 0.f;
    if (rr != 0 && rr != h) x = rr < h ? sv[rr + (rr >> 5)] : -sv[(Q - rr) + ((Q - rr) >> 5)];
    return x > 0.f ? x : 0.f;
  };
  double g;
  int sc;
  long long tot;
  warp_row_cdf(xres, Q, r0, n_M, log2_nM, lane, cdf ? cdf + (size_t)row * n_M : nullptr, g, sc, tot,
               gthr == nullptr,  // the step's rows (with thresholds) skip all-zero CDFs
               ccdf ? ccdf + (size_t)row * kCdfBlocks : nullptr);
  if (lane == 0) {
    gamma[row] = g;
    if (scale) scale[row] = sc;
    if (gthr) {
      const unsigned long long thr = g > 0.0 ? event_threshold(g, dt, flags) : 0ull;
      gthr[row] = thr;
      if (thr_cell) thr_cell[__ldg(occ + row)] = thr;
    }
  }
}

// gamma (and the scale s) alone, from the folded row: column r of the half
// period carries V_W at the cnt(r) grid momenta M = r (mod Q) and -V_W at the
// cnt(Q - r) momenta M = -r (mod Q).  The maximum over the grid and the sum of
// the quantised positive parts are the same integers the full CDF pass forms
// (same s, exact int64 sums), so gamma is bit-identical; the row is read once,
// coalesced, instead of once per grid column.
// number of M in [-n_M/2, n_M/2) with M = rr (mod Q), rr in [0, Q), for
// n_M = a Q + b and r0 = -n_M/2 mod Q: a, plus one where the grid's first b
// columns reach the residue
__device__ __forceinline__ int residue_count(int rr, int Q, int a, int b, int r0) {
  int off = rr - r0;
  if (off < 0) off += Q;
  return a + (off < b ? 1 : 0);
}

// C > 0: h <= 32 C, lane l holds the columns r = l + 32 c of a row and their
// two residue multiplicities in registers across the rows it visits; C = 0:
// any h, multiplicities formed per element.
template <int C>
__global__ __launch_bounds__(kCdfWarps * 32) void k_gamma_folded(int Q, int log2_nM, int ca, int cb, int r0,
                                                                 const float* __restrict__ VWh, int n_rows,
                                                                 double* __restrict__ gamma, int* __restrict__ scale) {
  const int lane = threadIdx.x & 31;
  const int h = Q / 2;
  constexpr int CR = C > 0 ? C : 1;
  int cp[CR], cn[CR];  // multiplicities of +V_W (residue r) and -V_W (residue Q - r)
#pragma unroll
  for (int c = 0; c < CR; ++c) {
    const int r = lane + 32 * c;
    const bool in = C > 0 && r >= 1 && r < h;
    cp[c] = in ? residue_count(r, Q, ca, cb, r0) : 0;
    cn[c] = in ? residue_count(Q - r, Q, ca, cb, r0) : 0;
  }
  for (int row = blockIdx.x * kCdfWarps + (threadIdx.x >> 5); row < n_rows; row += gridDim.x * kCdfWarps) {
    const float* v = VWh + (size_t)row * h;
    uint32_t mx = 0u;
    long long local = 0;
    if (C > 0) {
      float x[CR];
#pragma unroll
      for (int c = 0; c < CR; ++c) {
        const int r = lane + 32 * c;
        x[c] = r < h ? __ldg(v + r) : 0.f;
        const float xp = x[c] > 0.f && cp[c] ? x[c] : 0.f, xn = x[c] < 0.f && cn[c] ? -x[c] : 0.f;
        mx = max(mx, max(__float_as_uint(xp), __float_as_uint(xn)));
      }
      mx = __reduce_max_sync(0xffffffffu, mx);
      if (mx == 0u) {
        if (lane == 0) {
          gamma[row] = 0.0;
          if (scale) scale[row] = 0;
        }
        continue;
      }
      const int s = 61 - log2_nM - floor_log2_pos(__uint_as_float(mx));
#pragma unroll
      for (int c = 0; c < CR; ++c) {
        if (x[c] > 0.f) local += (long long)cp[c] * quantise(x[c], s);
        else if (x[c] < 0.f) local += (long long)cn[c] * quantise(-x[c], s);
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
      if (lane == 0) {
        gamma[row] = scaled_total(local, s);
        if (scale) scale[row] = s;
      }
    } else {
      for (int r = 1 + lane; r < h; r += 32) {
        const float x = __ldg(v + r);
        if (x > 0.f && residue_count(r, Q, ca, cb, r0) > 0) mx = max(mx, __float_as_uint(x));
        if (x < 0.f && residue_count(Q - r, Q, ca, cb, r0) > 0) mx = max(mx, __float_as_uint(-x));
      }
      mx = __reduce_max_sync(0xffffffffu, mx);
      if (mx == 0u) {
        if (lane == 0) {
          gamma[row] = 0.0;
          if (scale) scale[row] = 0;
        }
        continue;
      }
      const int s = 61 - log2_nM - floor_log2_pos(__uint_as_float(mx));
      for (int r = 1 + lane; r < h; r += 32) {
        const float x = __ldg(v + r);
        if (x > 0.f) local += (long long)residue_count(r, Q, ca, cb, r0) * quantise(x, s);
        else if (x < 0.f) local += (long long)residue_count(Q - r, Q, ca, cb, r0) * quantise(-x, s);
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
      if (lane == 0) {
        gamma[row] = scaled_total(local, s);
        if (scale) scale[row] = s;
      }
    }
  }
}

static int ceil_log2(int n) {
  int L = 0;
  while ((1 << L) < n) ++L;
  return L;
}

// ---------------------------------------------------------------- fused row kernel (h <= 128)
// For windows of up to 256 quadrature points one warp evaluates a whole kernel
// row: lane l owns the differences dV(m) for m = l + 1 + 32 q and the output
// columns r = l + 32 c; dV(m) is broadcast by shuffle and multiplied by the
// sine matrix staged in shared memory, with the same compensated (32-term
// chunk + TwoSum) FP32 accumulation as the tiled contraction.  When CDF
// outputs are given the warp then builds the row's fixed-point CDF, gamma and
// event threshold from the row it holds, saving a launch and a round trip.
constexpr int kRowWarps = 8;
constexpr int kRowMaxH = 128;

// A warp accumulates R rows together, sharing each sine load among them (R = 4
// when there are rows enough to fill the GPU that way, else 1).
template <int C, int R, int NET>  // output columns per lane: h <= 32 C; NET 1 or 2
__global__ __launch_bounds__(kRowWarps * 32) void k_kernel_rows_small(
    const float* __restrict__ V, int n_x, int bc, int Q, int n_M, int log2_nM, const int* __restrict__ occ,
    const int* __restrict__ n_occ_dev, int n_occ_host, const float* __restrict__ B, int Np, float c,
    float* __restrict__ VWh, long long* __restrict__ ccdf, int* __restrict__ scale, double* __restrict__ gamma,
    unsigned long long* __restrict__ gthr, unsigned long long* __restrict__ thr_cell, unsigned int* __restrict__ flags,
    double dt, const unsigned char* __restrict__ reach, DevHeader* __restrict__ hdr) {
  // reach != nullptr (one potential, occ == nullptr): row r is cell r, evaluated
  // only where the cell needs its kernel this step; the others get gamma = 0
  // and a zero event threshold
  extern __shared__ float s_mem[];
  const int h = Q / 2;
  const int Kt = NET == 1 ? h - 1 : h;  // terms of the contraction
  if (hdr && blockIdx.x == 0 && threadIdx.x == 0) hdr->rows_by_cell = reach ? 1u : 0u;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* s_B = s_mem;                                             // Kt x h, row = term
  float* s_row = s_mem + Kt * h + wid * (R + 1) * 32 * C;         // kernel row (h floats)
  float* s_dv = s_row + 32 * C;                                   // row g: dV(m) at s_dv[g 32 C + m - 1]
  const int n_rows = n_occ_dev ? *n_occ_dev : n_occ_host;
  if ((int)(blockIdx.x * kRowWarps * R) >= n_rows) return;
  // one pass over the rows (reach mode, the grid covers every row): each warp
  // loads its rows' reach bits and potential differences at once, before any
  // decision, and keeps them for the row loop
  const bool one_pass = reach && (int)(gridDim.x * kRowWarps * R) >= n_rows;
  unsigned row_ok = 0u;  // bit g: row g of this warp needs its kernel
  bool stage_B = true;
  if (one_pass) {
    float dv[R][C];
    bool any_ok = false, nz = false;
#pragma unroll
    for (int g = 0; g < R; ++g) {
      const int rw = (int)((blockIdx.x * kRowWarps + wid) * R) + g;
      if (rw < n_rows && cell_needs_kernel(reach, rw, n_x)) row_ok |= 1u << g;
#pragma unroll
      for (int q = 0; q < C; ++q) dv[g][q] = rw < n_rows ? a_term<NET>(V, n_x, bc, h, rw, lane + 32 * q) : 0.f;
    }
#pragma unroll
    for (int g = 0; g < R; ++g) {
      const bool okg = (row_ok >> g) & 1u;
      any_ok |= okg;
#pragma unroll
      for (int q = 0; q < C; ++q) {
        if (!okg) dv[g][q] = 0.f;
        nz |= dv[g][q] != 0.f;
        s_dv[g * 32 * C + lane + 32 * q] = dv[g][q];
      }
    }
    // a block none of whose cells needs a kernel only writes their zero
    // outputs; one whose needed cells all see a flat potential over the window
    // (their rows are exactly zero, the sums are skipped) needs no sine matrix
    if (!__syncthreads_or(any_ok)) {
      if (gamma && lane == 0) {
#pragma unroll
        for (int g = 0; g < R; ++g) {
          const int rw = (int)((blockIdx.x * kRowWarps + wid) * R) + g;
          if (rw < n_rows) {
            gamma[rw] = 0.0;
            gthr[rw] = 0ull;
            if (thr_cell) thr_cell[rw] = 0ull;
          }
        }
      }
      return;
    }
    stage_B = __syncthreads_or(nz);
  }
  if (stage_B) {
    // stage the sine rows with eight loads in flight per thread
    const int nB = Kt * h;
    for (int q0 = threadIdx.x; q0 < nB; q0 += 8 * kRowWarps * 32) {
      float tmp[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int q = q0 + u * kRowWarps * 32;
        const int m1 = q / h, r = q - m1 * h;
        tmp[u] = q < nB ? __ldg(B + (size_t)m1 * Np + r) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int q = q0 + u * kRowWarps * 32;
        if (q < nB) s_B[q] = tmp[u];
      }
    }
  }
  __syncthreads();
  const int r0 = ((-(n_M / 2)) % Q + Q) % Q;
  for (int row0 = (blockIdx.x * kRowWarps + wid) * R; row0 < n_rows; row0 += gridDim.x * kRowWarps * R) {
#pragma unroll
    for (int g = 0; g < R && !one_pass; ++g) {  // (one pass: loaded above)
      const int row = row0 + g;
      const bool ok = row < n_rows && (!reach || cell_needs_kernel(reach, row, n_x));
      const int i = ok ? (occ ? __ldg(occ + row) : row % n_x) : 0;
      const float* Vr = (occ || !ok) ? V : V + (size_t)(row / n_x) * n_x;
#pragma unroll
      for (int q = 0; q < C; ++q) s_dv[g * 32 * C + lane + 32 * q] = ok ? a_term<NET>(Vr, n_x, bc, h, i, lane + 32 * q) : 0.f;
    }
    bool nz = false;  // rows over a flat potential are exactly zero: skip the sums
#pragma unroll
    for (int g = 0; g < R; ++g)
#pragma unroll
      for (int q = 0; q < C; ++q) nz |= s_dv[g * 32 * C + lane + 32 * q] != 0.f;
    nz = __any_sync(0xffffffffu, nz);
    __syncwarp();
    float sacc[R][C], eacc[R][C];
#pragma unroll
    for (int g = 0; g < R; ++g)
#pragma unroll
      for (int cc = 0; cc < C; ++cc) sacc[g][cc] = eacc[g][cc] = 0.f;
    for (int j0 = 0; nz && j0 < Kt; j0 += 32) {   // chunks of 32 window terms
      float part[R][C];
#pragma unroll
      for (int g = 0; g < R; ++g)
#pragma unroll
        for (int cc = 0; cc < C; ++cc) part[g][cc] = 0.f;
      const int j1 = min(j0 + 32, Kt);
      for (int j = j0; j < j1; ++j) {
        const float* brow = s_B + j * h;
        float b[C];
#pragma unroll
        for (int cc = 0; cc < C; ++cc) {
          const int r = lane + 32 * cc;
          b[cc] = r < h ? brow[r] : 0.f;
        }
#pragma unroll
        for (int g = 0; g < R; ++g) {
          const float d = s_dv[g * 32 * C + j];
#pragma unroll
          for (int cc = 0; cc < C; ++cc) part[g][cc] = fmaf(d, b[cc], part[g][cc]);
        }
      }
#pragma unroll
      for (int g = 0; g < R; ++g)
#pragma unroll
        for (int cc = 0; cc < C; ++cc) two_sum_acc(sacc[g][cc], eacc[g][cc], part[g][cc]);
    }
#pragma unroll
    for (int g = 0; g < R; ++g) {
      const int row = row0 + g;
      if (row >= n_rows) break;
      if (reach && !(one_pass ? ((row_ok >> g) & 1u) != 0u : cell_needs_kernel(reach, row, n_x))) {
        if (gamma && lane == 0) {
          gamma[row] = 0.0;
          gthr[row] = 0ull;
          if (thr_cell) thr_cell[row] = 0ull;
        }
        continue;
      }
      float* out = VWh + (size_t)row * h;
#pragma unroll
      for (int cc = 0; cc < C; ++cc) {
        const int r = lane + 32 * cc;
        if (r < h) {
          const float v = __fmul_rn(c, __fadd_rn(sacc[g][cc], eacc[g][cc]));
          out[r] = v;
          s_row[r] = v;
        }
      }
      __syncwarp();
      if (gamma) {
        auto xres = [&](int rr) { return positive_part_smem(s_row, Q, rr); };
        double gm;
        int sc;
        long long tot;
        warp_row_cdf(xres, Q, r0, n_M, log2_nM, lane, nullptr, gm, sc, tot, false,
                     ccdf + (size_t)row * kCdfBlocks);
        if (lane == 0) {
          gamma[row] = gm;
          scale[row] = sc;
          const unsigned long long thr = gm > 0.0 ? event_threshold(gm, dt, flags) : 0ull;
          gthr[row] = thr;
          if (thr_cell) thr_cell[occ ? __ldg(occ + row) : row % n_x] = thr;
        }
      }
      __syncwarp();
    }
  }
}

bool small_window(const wmc_params& p) { return p.Q / 2 <= kRowMaxH; }

static size_t rows_small_smem(int h, int R, int net) {
  const int C = h <= 32 ? 1 : (h <= 64 ? 2 : 4);
  const int Kt = net == 2 ? h : h - 1;
  return sizeof(float) * ((size_t)Kt * h + (size_t)kRowWarps * (R + 1) * 32 * C);
}

cudaError_t launch_kernel_rows_small(const wmc_params& p, const float* V, const int* occ, const int* n_occ_dev,
                                     int n_occ_host, int max_rows, const float* B, float* VWh, long long* ccdf,
                                     int* scale, double* gamma, unsigned long long* gthr,
                                     unsigned long long* thr_cell, unsigned int* flags, cudaStream_t s,
                                     const unsigned char* reach, DevHeader* hdr, int net) {
  if (max_rows <= 0) return cudaSuccess;
  const Layout L = layout(p);
  const int h = L.h;
  const float c = (float)(-2.0 / (kHbarEVs * (double)p.Q));
  const int R = (long long)max_rows >= 2ll * num_sms() * kRowWarps * 4 ? 4 : 1;
  const size_t sm = rows_small_smem(h, R, net);
  int blocks = (max_rows + kRowWarps * R - 1) / (kRowWarps * R);
  if (blocks > 2 * num_sms()) blocks = 2 * num_sms();
  const int lg = ceil_log2(p.n_M);
#define WMC_LAUNCH_ROWS_NET(CC, RR, NN)                                                                           \
  do {                                                                                                            \
    if (sm > 48 * 1024)                                                                                           \
      raise_smem_limit(reinterpret_cast<const void*>(k_kernel_rows_small<CC, RR, NN>), sm);                   \
    k_kernel_rows_small<CC, RR, NN><<<blocks, kRowWarps * 32, sm, s>>>(                                           \
        V, p.n_x, p.bc_potential, p.Q, p.n_M, lg, occ, n_occ_dev, n_occ_host, B, L.Np, c, VWh, ccdf, scale,       \
        gamma, gthr, thr_cell, flags, p.dt_s, reach, hdr);                                                        \
  } while (0)
#define WMC_LAUNCH_ROWS(CC, RR)                     \
  do {                                              \
    if (net == 2) WMC_LAUNCH_ROWS_NET(CC, RR, 2);   \
    else WMC_LAUNCH_ROWS_NET(CC, RR, 1);            \
  } while (0)
  if (R == 4) {
    if (h <= 32) WMC_LAUNCH_ROWS(1, 4);
    else if (h <= 64) WMC_LAUNCH_ROWS(2, 4);
    else WMC_LAUNCH_ROWS(4, 4);
  } else {
    if (h <= 32) WMC_LAUNCH_ROWS(1, 1);
    else if (h <= 64) WMC_LAUNCH_ROWS(2, 1);
    else WMC_LAUNCH_ROWS(4, 1);
  }
#undef WMC_LAUNCH_ROWS
#undef WMC_LAUNCH_ROWS_NET
  return cudaGetLastError();
}


cudaError_t launch_cdf(const wmc_params& p, const float* VWh, const int* n_rows_dev, int n_rows_host, int max_rows,
                       long long* cdf, double* gamma, int* scale, unsigned long long* gthr, const int* occ,
                       unsigned long long* thr_cell, unsigned int* flags, cudaStream_t s, DevHeader* hdr,
                       long long* ccdf) {
  if (max_rows <= 0) return cudaSuccess;
  if (!cdf && !ccdf && !gthr && !n_rows_dev) {  // gamma (and scale) only
    const int h = p.Q / 2, ca = p.n_M / p.Q, cb = p.n_M - ca * p.Q, r0 = ((-(p.n_M / 2)) % p.Q + p.Q) % p.Q;
    int blocks = (max_rows + kCdfWarps - 1) / kCdfWarps;
    if (blocks > 8 * num_sms()) blocks = 8 * num_sms();
    const int lg = ceil_log2(p.n_M);
    if (h <= 32)
      k_gamma_folded<1><<<blocks, kCdfWarps * 32, 0, s>>>(p.Q, lg, ca, cb, r0, VWh, n_rows_host, gamma, scale);
    else if (h <= 64)
      k_gamma_folded<2><<<blocks, kCdfWarps * 32, 0, s>>>(p.Q, lg, ca, cb, r0, VWh, n_rows_host, gamma, scale);
    else if (h <= 128)
      k_gamma_folded<4><<<blocks, kCdfWarps * 32, 0, s>>>(p.Q, lg, ca, cb, r0, VWh, n_rows_host, gamma, scale);
    else
      k_gamma_folded<0><<<blocks, kCdfWarps * 32, 0, s>>>(p.Q, lg, ca, cb, r0, VWh, n_rows_host, gamma, scale);
    return cudaGetLastError();
  }
  const size_t sm = sizeof(float) * (size_t)kCdfWarps * (size_t)(p.Q / 2 + p.Q / 64 + 1);
  if (sm > 48 * 1024) {
    cudaError_t e = raise_smem_limit(reinterpret_cast<const void*>(k_cdf), sm);
    if (e != cudaSuccess) return e;
  }
  k_cdf<<<(max_rows + kCdfWarps - 1) / kCdfWarps, kCdfWarps * 32, sm, s>>>(
      p.n_M, p.Q, ceil_log2(p.n_M), VWh, n_rows_dev, n_rows_host, cdf, gamma, scale, gthr, occ, thr_cell, flags,
      p.dt_s, hdr, ccdf);
  return cudaGetLastError();
}

}  // namespace wmc

namespace wmc {

// ---------------------------------------------------------------- sliding-window evaluation (FP64)
// Eq. (wigner-1d-discrete) on every cell by a sliding window: for the
// half-period column r, E(l) = exp(i 2 pi l r / Q) and
//   W(i) = sum_{l=i-h}^{i+h} V(l) E(l),   VWh[i][r] = c Im[E(-i) W(i)],
// W(i + 1) = W(i) + V(i+h+1) E(i+h+1) - V(i-h) E(i-h).  One thread per
// (column, run of kDftSeg cells): the window sum at the run's first cell
// directly, then one slide per cell, all in FP64 with the exact integer
// phases l r mod Q (cos and sin of the Q phases staged in shared memory).
// Lanes take consecutive columns, so the potential loads are broadcasts and
// the row stores coalesce.
constexpr int kDftSeg = 256;

__global__ __launch_bounds__(256) void k_kernel_dft(const float* __restrict__ V, int n_x, int bc, int Q,
                                                    const double* __restrict__ CS, double c,
                                                    float* __restrict__ VWh) {
  extern __shared__ double s_cs[];  // [Q] cos, [Q] sin
  const int h = Q / 2;
  for (int q = threadIdx.x; q < 2 * Q; q += blockDim.x) s_cs[q] = CS[q];
  __syncthreads();
  const double* sC = s_cs;
  const double* sS = s_cs + Q;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = (int)(idx % h);
  const long long seg = idx / h;
  const long long i0 = seg * kDftSeg;
  if (i0 >= n_x) return;
  const long long i1 = i0 + kDftSeg < n_x ? i0 + kDftSeg : n_x;
  // W at i0
  double wr = 0.0, wi = 0.0;
  long long t = (((i0 - h) % Q) * r % Q + Q) % Q;
  for (long long l = i0 - h; l <= i0 + h; ++l) {
    const double v = (double)pot(V, n_x, bc, l);
    wr = fma(v, sC[t], wr);
    wi = fma(v, sS[t], wi);
    t += r;
    if (t >= Q) t -= Q;
  }
  long long ti = ((i0 % Q) * r) % Q;           // phase of E(i)
  long long ta = (((i0 + h + 1) % Q) * r) % Q;  // of E(i + h + 1)
  long long tb = ((((i0 - h) % Q + Q) % Q) * r) % Q;  // of E(i - h)
  for (long long i = i0; i < i1; ++i) {
    VWh[(size_t)i * h + r] = (float)(c * (sC[ti] * wi - sS[ti] * wr));
    const double va = (double)pot(V, n_x, bc, i + h + 1), vb = (double)pot(V, n_x, bc, i - h);
    wr += va * sC[ta] - vb * sC[tb];
    wi += va * sS[ta] - vb * sS[tb];
    ti += r;
    if (ti >= Q) ti -= Q;
    ta += r;
    if (ta >= Q) ta -= Q;
    tb += r;
    if (tb >= Q) tb -= Q;
  }
}

__global__ void k_dft_tables(int Q, double* __restrict__ CS) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < Q; t += gridDim.x * blockDim.x) {
    CS[t] = cospi(2.0 * (double)t / (double)Q);
    CS[Q + t] = sinpi(2.0 * (double)t / (double)Q);
  }
}

cudaError_t launch_kernel_dft(const wmc_params& p, const float* V, double* CS, float* VWh, cudaStream_t s) {
  const int h = p.Q / 2;
  k_dft_tables<<<(p.Q + 255) / 256, 256, 0, s>>>(p.Q, CS);
  const long long threads = (long long)h * ((p.n_x + kDftSeg - 1) / kDftSeg);
  const size_t sm = sizeof(double) * 2 * (size_t)p.Q;
  if (sm > 48 * 1024) {
    const cudaError_t e = raise_smem_limit(reinterpret_cast<const void*>(k_kernel_dft), sm);
    if (e != cudaSuccess) return e;
  }
  const double c = -2.0 / (kHbarEVs * (double)p.Q);
  k_kernel_dft<<<(unsigned)((threads + 255) / 256), 256, sm, s>>>(V, p.n_x, p.bc_potential, p.Q, CS, c, VWh);
  return cudaGetLastError();
}

}  // namespace wmc
