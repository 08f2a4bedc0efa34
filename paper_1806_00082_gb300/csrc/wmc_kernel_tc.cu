// Wigner-kernel contraction on the 5th-generation tensor cores (tcgen05):
// the precision forms of wmc_kernel_eval (BF16, FP16, FP16 hi/lo split).
//
//   VWh[row][r] = c * sum_{m=1}^{h-1} A[row][m] S[m][r],  A[row][m] = V(i+m) - V(i-m)
//
// One CTA of 128 threads computes a 128-row x 128-column output tile.  For each
// K block of 64 window terms:
//   - thread 0 starts bulk (TMA) copies of the precomputed sine-matrix operand
//     image(s) of this tile and K block into shared memory, completing on an
//     mbarrier;
//   - every thread builds its row of the A operand (64 potential differences,
//     rounded to the input type) in shared memory;
//   - after a proxy fence and a barrier, thread 0 issues four
//     tcgen05.mma (M = 128, N = 128, K = 16) per product into accumulators in
//     tensor memory and commits them to a second mbarrier, which every thread
//     waits on before the shared buffers are rewritten.
// Operands use the K-major layout without swizzle: 8-row x 16-byte core
// matrices, 128 bytes apart along K (LBO) and 1024 bytes apart along M/N (SBO).
// Accumulation: the main product is split over two K halves held in separate
// FP32 accumulators; the split form's cross terms (A_hi B_lo + A_lo B_hi, both
// lo parts scaled by 2^11) go to a third.  The epilogue reads them with
// tcgen05.ld and combines them in FP32.
//
// Every wait is bounded (about one second of SM clock); on a timeout the CTA
// sets WMC_FLAG_TIMEOUT, stops issuing work, and still frees its tensor memory.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "wmc_internal.cuh"

namespace wmc {

namespace {

constexpr int TM = 128, TN = 128, TK = 64;
constexpr uint32_t kLBO = 128, kSBO = 1024;
constexpr uint32_t kTileBytes = TN * TK * 2;  // one 128 x 64 16-bit operand image
constexpr long long kWaitCycles = 2000000000ll;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Waits for the phase of the given parity; false after about a second.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// K-major, no-swizzle shared-memory matrix descriptor (version 1).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(kLBO >> 4) << 16) | ((uint64_t)(kSBO >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor of kind::f16: D FP32, A and B of one 16-bit format
// (0 FP16, 1 BF16), both K-major, M = 128, N = 128.
__host__ __device__ constexpr uint32_t idesc_f16(uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 16 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ float potential_at(const float* __restrict__ V, int n_x, int bc, long long l) {
  if (l >= 0 && l < n_x) return __ldg(V + l);
  if (!bc) return 0.f;
  return __ldg(V + (l < 0 ? 0 : n_x - 1));
}

// Byte offset of element (row, k) of a 128 x 64 K-major core-matrix image.
__host__ __device__ __forceinline__ uint32_t core_offset(int row, int k) {
  return (uint32_t)((row >> 3) * kSBO + (k >> 3) * kLBO + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint16_t to_bits(float x, int prec) {
  if (prec == WMC_BF16) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
  return __half_as_ushort(__float2half_rn(x));
}

__device__ __forceinline__ float from_bits(uint16_t b, int prec) {
  if (prec == WMC_BF16) return __bfloat162float(__ushort_as_bfloat16(b));
  return __half2float(__ushort_as_half(b));
}

}  // namespace

// ---------------------------------------------------------------- operand images
// img[(nt * KB + kb)] is the 128 x 64 image of S[m = kb*64 + k + 1][r = nt*128 + n]
// (zero outside m < h, r < h), rounded to BF16 (img_bf16), FP16 (img_hi) and the
// FP16 residual scaled by 2^11 (img_lo).
__global__ void k_init_tc_images(int Q, int KB, int NT, uint16_t* __restrict__ img_bf16,
                                 uint16_t* __restrict__ img_hi, uint16_t* __restrict__ img_lo) {
  const int h = Q / 2;
  const long long total = (long long)NT * KB * TN * TK;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int blk = (int)(q / (TN * TK));
    const int e = (int)(q % (TN * TK));
    const int n = e / TK, k = e % TK;
    const int nt = blk / KB, kb = blk % KB;
    const int m = kb * TK + k + 1, r = nt * TN + n;
    float v = 0.f;
    if (m <= h - 1 && r < h) {
      const long long t = ((long long)m * r) % Q;
      v = __double2float_rn(sinpi(2.0 * (double)t / (double)Q));
    }
    const size_t off = (size_t)blk * (kTileBytes / 2) + core_offset(n, k) / 2;
    img_bf16[off] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
    const __half hi = __float2half_rn(v);
    img_hi[off] = __half_as_ushort(hi);
    img_lo[off] = __half_as_ushort(__float2half_rn((v - __half2float(hi)) * 2048.f));
  }
}

// ---------------------------------------------------------------- contraction
template <int PREC>
__global__ __launch_bounds__(128, 1) void k_kernel_eval_tc(const float* __restrict__ V, int n_x, int bc, int Q,
                                                           const int* __restrict__ occ,
                                                           const int* __restrict__ n_occ_dev, int n_occ_host,
                                                           const uint16_t* __restrict__ img_b,
                                                           const uint16_t* __restrict__ img_lo, int KB, float c,
                                                           float* __restrict__ VWh, unsigned int* __restrict__ flags) {
  constexpr bool SPLIT = PREC == WMC_FP16_SPLIT;
  constexpr int kind_fmt = PREC == WMC_BF16 ? 1 : 0;
  constexpr uint32_t kCols = SPLIT ? 512u : 256u;
  constexpr uint32_t idesc = idesc_f16(kind_fmt);
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sAhi = smem;
  uint8_t* sBhi = smem + kTileBytes;
  uint8_t* sAlo = smem + 2 * kTileBytes;  // split form only
  uint8_t* sBlo = smem + 3 * kTileBytes;
  __shared__ __align__(8) uint64_t bar_tma;
  __shared__ __align__(8) uint64_t bar_mma;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;

  const int n_rows = n_occ_dev ? *n_occ_dev : n_occ_host;
  const int row0 = blockIdx.x * TM, col0 = blockIdx.y * TN;
  const int h = Q / 2;
  if (row0 >= n_rows || col0 >= h) return;  // uniform over the CTA, before any allocation
  const int tid = threadIdx.x, warp = tid >> 5;

  if (warp == 0) tmem_alloc(&tmem_slot, kCols);
  if (tid == 0) {
    mbar_init(&bar_tma, 1);
    mbar_init(&bar_mma, 1);
    fence_mbar_init();
    s_abort = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t accA = tmem, accB = tmem + (uint32_t)TN, accX = tmem + 2u * (uint32_t)TN;

  const int my_row = row0 + tid;
  // occ == nullptr: implicit rows over consecutive potentials
  const int cell = my_row < n_rows ? (occ ? __ldg(occ + my_row) : my_row % n_x) : 0;
  const float* Vr = (occ || my_row >= n_rows) ? V : V + (size_t)(my_row / n_x) * n_x;
  const int half_kb = (KB + 1) / 2;
  const uint32_t tx_bytes = SPLIT ? 2u * kTileBytes : kTileBytes;
  // sine-matrix images of this column tile: the input-type (or FP16 hi) image
  // and, for the split form, the scaled FP16 residual image
  const uint16_t* imgB_tile = img_b + (size_t)blockIdx.y * KB * (kTileBytes / 2);
  const uint16_t* imgL_tile = SPLIT ? img_lo + (size_t)blockIdx.y * KB * (kTileBytes / 2) : nullptr;

  for (int kb = 0; kb < KB; ++kb) {
    if (tid == 0) {
      mbar_expect_tx(&bar_tma, tx_bytes);
      bulk_g2s(sBhi, imgB_tile + (size_t)kb * (kTileBytes / 2), kTileBytes, &bar_tma);
      if (SPLIT) bulk_g2s(sBlo, imgL_tile + (size_t)kb * (kTileBytes / 2), kTileBytes, &bar_tma);
    }
    // this thread's A row: 64 window terms m = kb*64 + k + 1
#pragma unroll
    for (int k8 = 0; k8 < TK / 8; ++k8) {
      uint32_t hw[4], lw[4];
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        uint16_t hb[2], lb[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int m = kb * TK + k8 * 8 + e + u + 1;
          float dv = 0.f;
          if (m <= h - 1 && my_row < n_rows)
            dv = __fsub_rn(potential_at(Vr, n_x, bc, (long long)cell + m), potential_at(Vr, n_x, bc, (long long)cell - m));
          hb[u] = to_bits(dv, SPLIT ? WMC_FP16 : PREC);
          if (SPLIT) lb[u] = to_bits(__fmul_rn(__fsub_rn(dv, from_bits(hb[u], WMC_FP16)), 2048.f), WMC_FP16);
        }
        hw[e / 2] = (uint32_t)hb[0] | ((uint32_t)hb[1] << 16);
        if (SPLIT) lw[e / 2] = (uint32_t)lb[0] | ((uint32_t)lb[1] << 16);
      }
      const uint32_t off = core_offset(tid, k8 * 8);
      *reinterpret_cast<uint4*>(sAhi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      if (SPLIT) *reinterpret_cast<uint4*>(sAlo + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      if (!mbar_wait(&bar_tma, (uint32_t)(kb & 1))) {
        atomicOr(flags, WMC_FLAG_TIMEOUT);
        s_abort = 1;
      } else {
        tc_fence_after();
        const uint32_t acc = kb < half_kb ? accA : accB;
        const int first = kb == 0 || kb == half_kb;
#pragma unroll
        for (int s = 0; s < TK / 16; ++s) {
          const uint64_t a_hi = smem_desc(smem_u32(sAhi) + s * 2 * kLBO);
          const uint64_t b_hi = smem_desc(smem_u32(sBhi) + s * 2 * kLBO);
          mma_f16(acc, a_hi, b_hi, idesc, (first && s == 0) ? 0u : 1u);
          if (SPLIT) {
            const uint64_t a_lo = smem_desc(smem_u32(sAlo) + s * 2 * kLBO);
            const uint64_t b_lo = smem_desc(smem_u32(sBlo) + s * 2 * kLBO);
            mma_f16(accX, a_hi, b_lo, idesc, (kb == 0 && s == 0) ? 0u : 1u);
            mma_f16(accX, a_lo, b_hi, idesc, 1u);
          }
        }
        mma_commit(&bar_mma);
        if (!mbar_wait(&bar_mma, (uint32_t)(kb & 1))) {
          atomicOr(flags, WMC_FLAG_TIMEOUT);
          s_abort = 1;
        }
      }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (s_abort) break;
  }

  if (!s_abort) {
    // epilogue: lane (warp 32 w + l) of TMEM holds tile row 32 w + l
    const int row = row0 + warp * 32 + (tid & 31);
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    const bool has_B = KB > half_kb;
    for (int cc = 0; cc < TN; cc += 16) {
      float a[16], b[16], x[16];
      tmem_ld16(accA + lane_base + (uint32_t)cc, a);
      if (has_B) tmem_ld16(accB + lane_base + (uint32_t)cc, b);
      if (SPLIT) tmem_ld16(accX + lane_base + (uint32_t)cc, x);
      if (row < n_rows) {
        float* out = VWh + (size_t)row * h + col0 + cc;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          if (col0 + cc + q >= h) break;
          float v = a[q];
          if (has_B) v = __fadd_rn(v, b[q]);
          if (SPLIT) v = __fadd_rn(v, __fmul_rn(x[q], 0x1p-11f));
          out[q] = __fmul_rn(c, v);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kCols);
}

// ---------------------------------------------------------------- host side
struct TcImages {
  int KB, NT;
  size_t bytes_per_image;  // NT * KB * kTileBytes
};

static TcImages tc_geometry(const wmc_params& p) {
  TcImages g;
  const int h = p.Q / 2;
  g.KB = (h - 1 + TK - 1) / TK;
  if (g.KB < 1) g.KB = 1;
  g.NT = (h + TN - 1) / TN;
  g.bytes_per_image = (size_t)g.NT * g.KB * kTileBytes;
  return g;
}

size_t tc_images_bytes(const wmc_params& p) { return 3 * tc_geometry(p).bytes_per_image; }

cudaError_t launch_init_tc_images(const wmc_params& p, void* images, cudaStream_t s) {
  const TcImages g = tc_geometry(p);
  uint16_t* base = static_cast<uint16_t*>(images);
  const size_t n16 = g.bytes_per_image / 2;
  k_init_tc_images<<<256, 256, 0, s>>>(p.Q, g.KB, g.NT, base, base + n16, base + 2 * n16);
  return cudaGetLastError();
}

cudaError_t launch_kernel_eval_tc(const wmc_params& p, int prec, const float* V, const int* occ, const int* n_occ_dev,
                                  int n_occ_host, int max_rows, const void* images, float* VWh, unsigned int* flags,
                                  cudaStream_t s) {
  if (max_rows <= 0) return cudaSuccess;
  const TcImages g = tc_geometry(p);
  const uint16_t* base = static_cast<const uint16_t*>(images);
  const size_t n16 = g.bytes_per_image / 2;
  const float c = (float)(-2.0 / (kHbarEVs * (double)p.Q));
  dim3 grid((max_rows + TM - 1) / TM, g.NT);
  if (prec == WMC_BF16) {
    const size_t sm = 2 * kTileBytes;
    k_kernel_eval_tc<WMC_BF16><<<grid, 128, sm, s>>>(V, p.n_x, p.bc_potential, p.Q, occ, n_occ_dev, n_occ_host,
                                                     base, nullptr, g.KB, c, VWh, flags);
  } else if (prec == WMC_FP16) {
    const size_t sm = 2 * kTileBytes;
    k_kernel_eval_tc<WMC_FP16><<<grid, 128, sm, s>>>(V, p.n_x, p.bc_potential, p.Q, occ, n_occ_dev, n_occ_host,
                                                     base + n16, nullptr, g.KB, c, VWh, flags);
  } else if (prec == WMC_FP16_SPLIT) {
    const size_t sm = 4 * kTileBytes;
    cudaFuncSetAttribute(k_kernel_eval_tc<WMC_FP16_SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_kernel_eval_tc<WMC_FP16_SPLIT><<<grid, 128, sm, s>>>(V, p.n_x, p.bc_potential, p.Q, occ, n_occ_dev,
                                                           n_occ_host, base + n16, base + 2 * n16, g.KB, c, VWh,
                                                           flags);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace wmc
