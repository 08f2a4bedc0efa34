// Wigner-kernel contraction on the 5th-generation tensor cores (tcgen05):
// the precision forms of wmc_kernel_eval (BF16, FP16, FP16 hi/lo split, 3xTF32).
//
//   VWh[row][r] = c * sum_{m=1}^{h-1} A[row][m] S[m][r],  A[row][m] = V(i+m) - V(i-m)
//
// The sine matrix S is precomputed once per workspace as operand images in
// global memory (BF16, FP16 hi, FP16 lo, TF32 hi, TF32 lo) in 16 KB blocks of
// 128 rows in the layout below; A is generated on chip from the potential
// and never written to global memory.  Three kernels:
//   - k_kernel_eval_tc_ta<BF16 | FP16, N>: warp-specialised (16 builder /
//     epilogue warps, one MMA-issuing thread, one bulk-copy thread), the whole
//     A operand of a 128-row tile in tensor memory, B streamed through a deep
//     ring of shared-memory stages, M = N = 128, two TMEM accumulator buffers
//     so that the epilogue of one column tile overlaps the MMAs of the next
//     (K <= 512);
//   - k_kernel_eval_tc_ws_split<FP16 | TF32>: the hi/lo split forms, three MMAs
//     per K step (hi x hi, hi x lo, lo x hi), A resident in shared memory per
//     K pass, each K block's main product in its own accumulator;
//   - k_kernel_eval_tc: a per-tile kernel with both operands streamed, for
//     BF16 / FP16 windows wider than the tensor-memory form holds.
// Shared-memory operands use the K-major 128-byte swizzled layout: rows of
// 128 bytes (64 16-bit or 32 TF32 values), 8-row atoms 1024 bytes apart, the
// 16-byte chunks of row r XOR-swizzled by r % 8; shared-memory blocks are
// aligned to 1024 bytes.  Accumulation is FP32 in TMEM; the epilogue reads
// the accumulators with tcgen05.ld and combines and scales them in FP32.
//
// Every wait is bounded (about one second of SM clock); on a timeout the CTA
// sets WMC_FLAG_TIMEOUT, stops issuing work, lets its copies and MMAs in
// flight complete (bounded again) and still frees its tensor memory.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "wmc_device.cuh"

namespace wmc {

namespace {

constexpr int TM = 128, TN = 128, TK = 64;
constexpr uint32_t kSBO = 1024, kKStepBytes = 32;  // atom stride; bytes per K step of 16
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

// One probe of the phase of the given parity.  While the phase is incomplete
// the thread may sleep in hardware for up to kSuspendNs nanoseconds (woken
// when the phase completes) instead of spinning on the barrier word.
constexpr uint32_t kSuspendNs = 100000;
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
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

// K-major shared-memory matrix descriptor (version 1) of the 128-byte swizzled
// layout: 8-row atoms of 128-byte rows (64 16-bit K values) 1024 bytes apart
// (SBO), the 16-byte chunks of row r XOR-swizzled by r % 8; a K step of 16
// values advances the start address by 32 bytes inside the atom.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)(kSBO >> 4) << 32) | (1ull << 46) |
         (2ull << 61);
}

// Dynamic shared memory rounded up to the 1024-byte alignment the swizzled
// atoms need (launches request kSmemAlignPad extra bytes).
constexpr uint32_t kSmemAlignPad = 1024;
__device__ __forceinline__ uint8_t* align_smem(uint8_t* p) {
  const uint32_t a = smem_u32(p);
  return p + (((a + 1023u) & ~1023u) - a);
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

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// x rounded to TF32 (nearest, ties away from zero), as FP32 bits with the low
// 13 mantissa bits zero.
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_wait16(uint32_t* r);

// 16 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  tmem_wait16(r);
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// Split form of tmem_ld16: the load is issued into r, and tmem_wait16 waits
// for all loads in flight while naming r as read-write, so that no use of r
// can be scheduled before the wait.
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait16(uint32_t* r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}

// 16 consecutive 32-bit columns of this thread's TMEM lane from registers;
// tmem_wait_st waits until this thread's stores are complete.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// kind::f16 MMA with the A operand in tensor memory: M = 128 rows in the 128
// lanes, each 32-bit column holding two consecutive K values (the lower K in
// the low half), K = 16 over 8 columns starting at a_tmem.
__device__ __forceinline__ void mma_f16_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ float potential_at(const float* __restrict__ V, int n_x, int bc, long long l) {
  if (l >= 0 && l < n_x) return __ldg(V + l);
  if (!bc) return 0.f;
  return __ldg(V + (l < 0 ? 0 : n_x - 1));
}

// Entry (row, kk) of the A operand: the N = 1 network's potential difference
// V(i + m) - V(i - m), m = kk + 1 (zero beyond m = h - 1), or the N = 2
// network's signed pair sum at offset u = kk: V(i+u) + V(i+u+1) if i + u is
// even, else -(V(i-u-1) + V(i-u)) (zero beyond u = h - 1).  From a staged
// window w (w[h + j] = V(i + j)) or from the potential itself.
template <int NET>
__device__ __forceinline__ float a_entry_window(const float* w, int h, int i, int kk) {
  if (NET == 1) {
    const int m = kk + 1;
    return m <= h - 1 ? __fsub_rn(w[h + m], w[h - m]) : 0.f;
  }
  const int u = kk;
  if (u > h - 1) return 0.f;
  return ((i + u) & 1) == 0 ? __fadd_rn(w[h + u], w[h + u + 1]) : -__fadd_rn(w[h - u - 1], w[h - u]);
}

// Byte offset of element (row, k) of a 128 x 64 K-major operand block in the
// 128-byte swizzled layout (row r at 128 r, chunk k / 8 stored at chunk
// (k / 8) ^ (r % 8)); blocks of consecutive rows concatenate.
__host__ __device__ __forceinline__ uint32_t core_offset(int row, int k) {
  return (uint32_t)(row * 128 + ((((k >> 3) ^ (row & 7)) & 7) << 4) + (k & 7) * 2);
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
                                 uint16_t* __restrict__ img_hi, uint16_t* __restrict__ img_lo, int net) {
  const long long total = (long long)NT * KB * TN * TK;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int blk = (int)(q / (TN * TK));
    const int e = (int)(q % (TN * TK));
    const int n = e / TK, k = e % TK;
    const int nt = blk / KB, kb = blk % KB;
    const int kk = kb * TK + k, r = nt * TN + n;
    const float v = net == 2 ? sine_entry_n2(Q, kk, r) : sine_entry_n1(Q, kk, r);
    const size_t off = (size_t)blk * (kTileBytes / 2) + core_offset(n, k) / 2;
    img_bf16[off] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
    const __half hi = __float2half_rn(v);
    img_hi[off] = __half_as_ushort(hi);
    img_lo[off] = __half_as_ushort(__float2half_rn((v - __half2float(hi)) * 2048.f));
  }
}

// The same sine matrix as TF32 hi/lo pairs (hi = tf32(v), lo = tf32(v - hi)),
// in 128 x 32 blocks of the swizzled layout (four 4-byte values per chunk).
__global__ void k_init_tc_images32(int Q, int KB32, int NT, uint32_t* __restrict__ img_hi,
                                   uint32_t* __restrict__ img_lo, int transposed) {
  const long long total = (long long)NT * KB32 * TN * 32;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int blk = (int)(q / (TN * 32));
    const int e = (int)(q % (TN * 32));
    const int n = e / 32, k = e % 32;
    const int nt = blk / KB32, kb = blk % KB32;
    // transposed (the adjoint's B): S[m][r] at n = m - 1, k = r
    const float v = transposed ? sine_entry_n1(Q, nt * TN + n, kb * 32 + k) : sine_entry_n1(Q, kb * 32 + k, nt * TN + n);
    // chunk k / 4 of row n, value k % 4 in it
    const size_t off = (size_t)blk * (kTileBytes / 4) + (core_offset(n, (k >> 2) * 8) >> 2) + (k & 3);
    const uint32_t hi = to_tf32(v);
    img_hi[off] = hi;
    img_lo[off] = to_tf32(v - __uint_as_float(hi));
  }
}

// ---------------------------------------------------------------- contraction
// Two pipeline stages: while the tensor cores run the MMAs of K block kb from
// stage kb % 2, the threads build the A operand of block kb + 1 into the other
// stage and thread 0 has already started the copy of its B operand(s); a
// stage is rewritten only after the MMAs that read it have completed (one
// mbarrier per stage for the copies, one for the MMA commits).  When the
// tile's 128 rows are 128 consecutive cells of one potential, the potential
// window they need is staged in shared memory once and the A operand is built
// from it without branches.
constexpr int kStages = 2;

__host__ __device__ constexpr size_t tc_smem_bytes(bool split, int h) {
  return kSmemAlignPad + (size_t)(split ? 8 : 4) * kTileBytes + sizeof(float) * (size_t)(TM + 2 * h);
}

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
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = align_smem(smem_raw);
  uint8_t* sA[kStages] = {smem, smem + kTileBytes};
  uint8_t* sB[kStages] = {smem + 2 * kTileBytes, smem + 3 * kTileBytes};
  uint8_t* sAl[kStages] = {smem + 4 * kTileBytes, smem + 5 * kTileBytes};  // split form only
  uint8_t* sBl[kStages] = {smem + 6 * kTileBytes, smem + 7 * kTileBytes};
  float* sV = reinterpret_cast<float*>(smem + (SPLIT ? 8 : 4) * kTileBytes);
  __shared__ __align__(8) uint64_t bar_tma[kStages];
  __shared__ __align__(8) uint64_t bar_mma[kStages];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort, s_cell0;

  const int n_rows = n_occ_dev ? *n_occ_dev : n_occ_host;
  const int row0 = blockIdx.x * TM, col0 = blockIdx.y * TN;
  const int h = Q / 2;
  if (row0 >= n_rows || col0 >= h) return;  // uniform over the CTA, before any allocation
  const int tid = threadIdx.x, warp = tid >> 5;

  if (warp == 0) tmem_alloc(&tmem_slot, kCols);
  if (tid == 0) {
    for (int q = 0; q < kStages; ++q) {
      mbar_init(&bar_tma[q], 1);
      mbar_init(&bar_mma[q], 1);
    }
    fence_mbar_init();
    s_abort = 0;
  }

  // this thread's row: occ == nullptr means implicit rows over consecutive
  // potentials (row r is cell r % n_x of potential r / n_x)
  const int my_row = row0 + tid;
  const bool valid = my_row < n_rows;
  const int cell = valid ? (occ ? __ldg(occ + my_row) : my_row % n_x) : 0;
  const int pot_idx = (occ || !valid) ? 0 : my_row / n_x;
  const float* Vr = V + (size_t)pot_idx * n_x;
  if (tid == 0) s_cell0 = cell;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t accA = tmem, accB = tmem + (uint32_t)TN, accX = tmem + 2u * (uint32_t)TN;
  const int pot0 = (occ || row0 >= n_rows) ? 0 : row0 / n_x;
  const bool contig = __syncthreads_and(valid && cell == s_cell0 + tid && pot_idx == pot0) != 0;
  if (contig) {
    const float* V0 = V + (size_t)pot0 * n_x;
    for (int q = tid; q < TM + 2 * h; q += blockDim.x) sV[q] = potential_at(V0, n_x, bc, (long long)s_cell0 - h + q);
  }

  const int half_kb = (KB + 1) / 2;
  const uint32_t tx_bytes = SPLIT ? 2u * kTileBytes : kTileBytes;
  const uint16_t* imgB_tile = img_b + (size_t)blockIdx.y * KB * (kTileBytes / 2);
  const uint16_t* imgL_tile = SPLIT ? img_lo + (size_t)blockIdx.y * KB * (kTileBytes / 2) : nullptr;

  auto issue_copy = [&](int kb, int st) {
    mbar_expect_tx(&bar_tma[st], tx_bytes);
    bulk_g2s(sB[st], imgB_tile + (size_t)kb * (kTileBytes / 2), kTileBytes, &bar_tma[st]);
    if (SPLIT) bulk_g2s(sBl[st], imgL_tile + (size_t)kb * (kTileBytes / 2), kTileBytes, &bar_tma[st]);
  };
  // this thread's A row of K block kb: window terms m = kb*64 + k + 1
  auto build_A = [&](int kb, int st) {
    if (contig) __syncthreads();  // the window is staged (first use) / keeps warps aligned
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
          if (m <= h - 1) {
            if (contig) dv = __fsub_rn(sV[tid + h + m], sV[tid + h - m]);
            else if (valid)
              dv = __fsub_rn(potential_at(Vr, n_x, bc, (long long)cell + m), potential_at(Vr, n_x, bc, (long long)cell - m));
          }
          hb[u] = to_bits(dv, SPLIT ? WMC_FP16 : PREC);
          if (SPLIT) lb[u] = to_bits(__fmul_rn(__fsub_rn(dv, from_bits(hb[u], WMC_FP16)), 2048.f), WMC_FP16);
        }
        hw[e / 2] = (uint32_t)hb[0] | ((uint32_t)hb[1] << 16);
        if (SPLIT) lw[e / 2] = (uint32_t)lb[0] | ((uint32_t)lb[1] << 16);
      }
      const uint32_t off = core_offset(tid, k8 * 8);
      *reinterpret_cast<uint4*>(sA[st] + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      if (SPLIT) *reinterpret_cast<uint4*>(sAl[st] + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
  };

  if (tid == 0) issue_copy(0, 0);
  build_A(0, 0);
  for (int kb = 0; kb < KB; ++kb) {
    const int st = kb & 1;
    const uint32_t ph = (uint32_t)((kb >> 1) & 1);
    fence_proxy_async_smem();
    __syncthreads();  // A of block kb is in stage st
    if (s_abort) break;
    if (tid == 0) {
      if (!mbar_wait(&bar_tma[st], ph)) {
        atomicOr(flags, WMC_FLAG_TIMEOUT);
        s_abort = 1;
      } else {
        tc_fence_after();
        const uint32_t acc = kb < half_kb ? accA : accB;
        const int first = kb == 0 || kb == half_kb;
#pragma unroll
        for (int s = 0; s < TK / 16; ++s) {
          const uint64_t a_hi = smem_desc(smem_u32(sA[st]) + s * kKStepBytes);
          const uint64_t b_hi = smem_desc(smem_u32(sB[st]) + s * kKStepBytes);
          mma_f16(acc, a_hi, b_hi, idesc, (first && s == 0) ? 0u : 1u);
          if (SPLIT) {
            const uint64_t a_lo = smem_desc(smem_u32(sAl[st]) + s * kKStepBytes);
            const uint64_t b_lo = smem_desc(smem_u32(sBl[st]) + s * kKStepBytes);
            mma_f16(accX, a_hi, b_lo, idesc, (kb == 0 && s == 0) ? 0u : 1u);
            mma_f16(accX, a_lo, b_hi, idesc, 1u);
          }
        }
        mma_commit(&bar_mma[st]);
        // the other stage is free once the MMAs of block kb - 1 are done
        if (kb + 1 < KB) {
          if (kb >= 1 && !mbar_wait(&bar_mma[st ^ 1], (uint32_t)(((kb - 1) >> 1) & 1))) {
            atomicOr(flags, WMC_FLAG_TIMEOUT);
            s_abort = 1;
          } else {
            issue_copy(kb + 1, st ^ 1);
          }
        }
      }
    }
    if (kb + 1 < KB) {
      if (kb >= 1 && !mbar_wait(&bar_mma[st ^ 1], (uint32_t)(((kb - 1) >> 1) & 1))) s_abort = 1;
      build_A(kb + 1, st ^ 1);
    }
  }
  // all MMAs of the tile done (commits complete in order)
  if (tid == 0 && !s_abort && !mbar_wait(&bar_mma[(KB - 1) & 1], (uint32_t)(((KB - 1) >> 1) & 1))) {
    atomicOr(flags, WMC_FLAG_TIMEOUT);
    s_abort = 1;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

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

// ---------------------------------------------------------------- warp-specialised forms
// Roles of the warp-specialised kernels below (576 threads): warps 0-15 build
// the A operand and then run the epilogue, warp 16 has one thread issue the
// MMAs, warp 17 one thread stream the B operand images.  The epilogue warp w
// reads TMEM lane quadrant w % 4 and transposes each 32 x 16 piece through
// shared memory, so that global stores are whole 64-byte row segments.
constexpr int kWsBuilders = 512;
constexpr int kWsThreads = kWsBuilders + 64;

constexpr int kWsStageFloats = 32 * 16;  // epilogue staging per warp: 32 rows x 16 columns

// AND of pred over the kWsBuilders builder threads (named barrier 1).
__device__ __forceinline__ bool builders_and(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred q, p;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "barrier.cta.red.and.pred p, 1, %2, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)pred), "n"(kWsBuilders)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void builders_sync() { asm volatile("barrier.cta.sync 1, %0;" ::"n"(kWsBuilders) : "memory"); }

template <int PREC>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
  if (PREC == WMC_BF16) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&v);
  } else {
    const __half2 v = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&v);
  }
}

// ---------------------------------------------------------------- A in tensor memory
// BF16 / FP16, K <= 512: one CTA per 128 rows and a run of 128-column tiles.
// The whole A operand of the row tile lives in tensor memory (up to 8 blocks
// of 64 K values, 32 columns each, at columns 0 .. 255), built once and used
// by every column tile; two 128-column FP32 accumulator buffers at columns
// 256 and 384 let the epilogue of tile j overlap the MMAs of tile j + 1; the
// shared memory holds a ring of 11 B stages (one 128-column x 64-K image
// each), so the tensor core reads only B from shared memory and the ring
// covers a copy round trip.  Builder warp w writes TMEM lanes 32 (w % 4) ..
// + 31 (one row of the tile per thread) for the K blocks kb = w / 4 (mod 4):
// its row's entries, packed in pairs, by tcgen05.st, then arrives on
// a_ready[kb].  The MMA thread waits for a_ready (first tile), each B stage
// and a drained accumulator buffer, commits each stage and each tile.  Every
// wait is bounded; on a timeout an abort flag makes all roles drain to the
// final barrier, after which TMEM is freed.
constexpr int kTaStages = 11;
constexpr int kTaMaxKB = 8;
constexpr uint32_t kTaAccCol = 256;

__host__ __device__ constexpr size_t ta_smem_bytes(int h) {
  return kSmemAlignPad + (size_t)kTaStages * kTileBytes +
         sizeof(float) * (size_t)((TM + 2 * h) > (kWsBuilders / 32) * kWsStageFloats
                                      ? (TM + 2 * h)
                                      : (kWsBuilders / 32) * kWsStageFloats);
}

template <int PREC, int NET>
__global__ __launch_bounds__(kWsThreads, 1) void k_kernel_eval_tc_ta(const float* __restrict__ V, int n_x, int bc,
                                                                     int Q, const int* __restrict__ occ,
                                                                     const int* __restrict__ n_occ_dev, int n_occ_host,
                                                                     const uint16_t* __restrict__ img_b, int KB,
                                                                     int NT, int n_split, float c,
                                                                     float* __restrict__ VWh,
                                                                     unsigned int* __restrict__ flags) {
  constexpr uint32_t idesc = idesc_f16(PREC == WMC_BF16 ? 1u : 0u);  // M = N = 128
  constexpr int STG = kTaStages;
  constexpr uint32_t n_cols = 512;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = align_smem(smem_raw);
  uint8_t* sB = smem;                                                     // STG stages of 128 x 64
  float* sV = reinterpret_cast<float*>(sB + (size_t)STG * kTileBytes);  // window, then epilogue staging
  __shared__ __align__(8) uint64_t a_ready[kTaMaxKB];
  __shared__ __align__(8) uint64_t b_full[kTaStages], b_empty[kTaStages];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2];
  __shared__ __align__(8) uint64_t drain;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;

  const int n_rows = n_occ_dev ? *n_occ_dev : n_occ_host;
  const int row0 = blockIdx.x * TM;
  const int h = Q / 2;
  if (row0 >= n_rows) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // this CTA's 128-column tiles: [nt_begin, nt_begin + n_my)
  const int nt_begin = (int)(((long long)blockIdx.y * NT) / n_split);
  const int n_my = (int)(((long long)(blockIdx.y + 1) * NT) / n_split) - nt_begin;
  const int n_tiles = n_my * KB;

  if (warp == 0) tmem_alloc(&tmem_slot, n_cols);
  if (tid == 0) {
    for (int q = 0; q < KB; ++q) mbar_init(&a_ready[q], 4);  // one arrival per lane-quarter warp
    for (int q = 0; q < STG; ++q) {
      mbar_init(&b_full[q], 1);
      mbar_init(&b_empty[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&acc_full[q], 1);
      mbar_init(&acc_empty[q], kWsBuilders / 32);  // one arrival per epilogue warp
    }
    mbar_init(&drain, 1);
    fence_mbar_init();
    s_abort = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == kWsBuilders / 32 + 1) {
    // ---- B producer
    if (lane == 0) {
      int issued = 0;
      for (int t = 0; t < n_tiles && !s_abort; ++t) {
        const int st = t % STG;
        if (t >= STG && !mbar_wait(&b_empty[st], (uint32_t)(((t / STG) - 1) & 1))) {
          atomicOr(flags, WMC_FLAG_TIMEOUT);
          s_abort = 1;
          break;
        }
        const int nt = nt_begin + t / KB, kb = t % KB;
        mbar_expect_tx(&b_full[st], kTileBytes);
        bulk_g2s(sB + (size_t)st * kTileBytes, img_b + ((size_t)nt * KB + kb) * (kTileBytes / 2), kTileBytes,
                 &b_full[st]);
        issued = t + 1;
      }
      if (s_abort)  // let the copies still in flight land before the CTA exits (bounded)
        for (int t = max(0, issued - STG); t < issued; ++t)
          (void)mbar_wait(&b_full[t % STG], (uint32_t)((t / STG) & 1));
    }
  } else if (warp == kWsBuilders / 32) {
    // ---- MMA issuer
    if (lane == 0) {
      for (int j = 0; j < n_my && !s_abort; ++j) {
        const int buf = j & 1;
        if (j >= 2 && !mbar_wait(&acc_empty[buf], (uint32_t)(((j - 2) >> 1) & 1))) {
          atomicOr(flags, WMC_FLAG_TIMEOUT);
          s_abort = 1;
          break;
        }
        tc_fence_after();
        const uint32_t acc = tmem + kTaAccCol + (uint32_t)(buf * TN);
        for (int kb = 0; kb < KB; ++kb) {
          const int t = j * KB + kb, st = t % STG;
          if ((j == 0 && !mbar_wait(&a_ready[kb], 0u)) ||
              !mbar_wait(&b_full[st], (uint32_t)((t / STG) & 1))) {
            atomicOr(flags, WMC_FLAG_TIMEOUT);
            s_abort = 1;
            break;
          }
          tc_fence_after();
          const uint32_t b_base = smem_u32(sB + (size_t)st * kTileBytes);
#pragma unroll
          for (int s4 = 0; s4 < TK / 16; ++s4)
            mma_f16_ta(acc, tmem + (uint32_t)(kb * (TK / 2) + s4 * 8), smem_desc(b_base + s4 * kKStepBytes), idesc,
                       (kb == 0 && s4 == 0) ? 0u : 1u);
          mma_commit(&b_empty[st]);
        }
        if (s_abort) break;
        mma_commit(&acc_full[buf]);
      }
      if (s_abort) {  // drain the MMAs already issued before TMEM is freed (bounded)
        mma_commit(&drain);
        (void)mbar_wait(&drain, 0u);
      }
    }
  } else {
    // ---- A builders (warps 0-15), then the epilogue
    // contiguity of the tile's rows (row row0 + tid % 128, each checked by four threads)
    const int rc = tid & (TM - 1);
    const int rowc = row0 + rc;
    const bool validc = rowc < n_rows;
    const int cellc = validc ? (occ ? __ldg(occ + rowc) : rowc % n_x) : 0;
    const int potc = (occ || !validc) ? 0 : rowc / n_x;
    const int cell0 = occ ? __ldg(occ + row0) : row0 % n_x;
    const int pot0 = occ ? 0 : row0 / n_x;
    const bool contig = builders_and(validc && cellc == cell0 + rc && potc == pot0);
    if (contig) {
      const float* V0 = V + (size_t)pot0 * n_x;
      constexpr int kU = 4;  // loads issued together
      for (int q0 = tid; q0 < TM + 2 * h; q0 += kU * kWsBuilders) {
        float v[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int q = q0 + u * kWsBuilders;
          v[u] = q < TM + 2 * h ? potential_at(V0, n_x, bc, (long long)cell0 - h + q) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u)
          if (q0 + u * kWsBuilders < TM + 2 * h) sV[q0 + u * kWsBuilders] = v[u];
      }
      builders_sync();
    }
    // this thread's row of the tile = its TMEM lane
    const int quad = warp & 3, kp = warp >> 2;
    const int rr = 32 * quad + lane;
    const int row = row0 + rr;
    const bool valid = row < n_rows;
    const int cell = (contig || !valid) ? 0 : (occ ? __ldg(occ + row) : row % n_x);
    const float* Vr = V + (size_t)((occ || !valid) ? 0 : row / n_x) * n_x;
    const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
#pragma unroll 1
    for (int kb = kp; kb < KB; kb += 4) {
      uint32_t wv[32];
      const int k0 = kb * TK;  // K index of the block's first value
      if (NET == 1 && contig && k0 + TK <= h - 1) {
        // m = k0 + 1 .. k0 + 64, all inside the sum: wp[m] = V(i + m), wp[-m] = V(i - m)
        const float* wp = sV + rr + h;
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          const int m = k0 + 2 * e + 1;
          wv[e] = pack2<PREC>(__fsub_rn(wp[m], wp[-m]), __fsub_rn(wp[m + 1], wp[-m - 1]));
        }
      } else {
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          const int kk = k0 + 2 * e;
          float a = 0.f, b = 0.f;
          if (contig) {
            a = a_entry_window<NET>(sV + rr, h, cell0 + rr, kk);
            b = a_entry_window<NET>(sV + rr, h, cell0 + rr, kk + 1);
          } else if (valid) {
            a = a_term<NET>(Vr, n_x, bc, h, cell, kk);
            b = a_term<NET>(Vr, n_x, bc, h, cell, kk + 1);
          }
          wv[e] = pack2<PREC>(a, b);
        }
      }
      tmem_st16(tmem + lane_base + (uint32_t)(kb * (TK / 2)), wv);
      tmem_st16(tmem + lane_base + (uint32_t)(kb * (TK / 2) + 16), wv + 16);
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&a_ready[kb])) : "memory");
    }
    // epilogue of each column tile: warp w reads lanes 32 (w % 4) .. + 31, columns 32 (w / 4) .. + 31
    const int cq = warp >> 2;
    float* stg = sV + warp * kWsStageFloats;
    const bool vec_ok = (h & 3) == 0 && (reinterpret_cast<uintptr_t>(VWh) & 15) == 0;
    for (int j = 0; j < n_my; ++j) {
      const int buf = j & 1;
      // lane 0 waits for the tile; the decision is warp-uniform because the
      // TMEM loads below are warp-collective
      int okw = 1;
      if (lane == 0) okw = !s_abort && mbar_wait(&acc_full[buf], (uint32_t)((j >> 1) & 1));
      const bool ok = __shfl_sync(0xffffffffu, okw, 0) != 0;
      if (!ok) {
        if (lane == 0) atomicOr(flags, WMC_FLAG_TIMEOUT);
        s_abort = 1;
        break;
      }
      tc_fence_after();
      constexpr int NP = TN / 64;  // pieces of 16 columns per warp
      uint32_t rg2[2][16];
      const uint32_t tbase = tmem + kTaAccCol + (uint32_t)(buf * TN) + lane_base + (uint32_t)(cq * (TN / 4));
      tmem_ld16_issue(tbase, rg2[0]);
      tmem_wait16(rg2[0]);
#pragma unroll
      for (int hf = 0; hf < NP; ++hf) {
        if (hf + 1 < NP) tmem_ld16_issue(tbase + (uint32_t)((hf + 1) * 16), rg2[(hf + 1) & 1]);
        const uint32_t* a = rg2[hf & 1];
        const int col0 = (nt_begin + j) * TN + cq * (TN / 4) + hf * 16;
        // row `lane` of the piece; its four 16-byte groups are XOR-swizzled by
        // (row / 2) % 4, so that the row-wise writes and the group-wise reads
        // below are free of bank conflicts
#pragma unroll
        for (int g = 0; g < 4; ++g)
          *reinterpret_cast<float4*>(stg + lane * 16 + 4 * (g ^ ((lane >> 1) & 3))) =
              make_float4(__fmul_rn(c, __uint_as_float(a[4 * g])), __fmul_rn(c, __uint_as_float(a[4 * g + 1])),
                          __fmul_rn(c, __uint_as_float(a[4 * g + 2])), __fmul_rn(c, __uint_as_float(a[4 * g + 3])));
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r2 = 8 * i + (lane >> 2), g = lane & 3;
          const float4 v = *reinterpret_cast<const float4*>(stg + r2 * 16 + 4 * (g ^ ((r2 >> 1) & 3)));
          const int grow = row0 + quad * 32 + r2, gcol = col0 + 4 * g;
          if (grow < n_rows && gcol < h) {
            float* out = VWh + (size_t)grow * h + gcol;
            if (vec_ok) {
              *reinterpret_cast<float4*>(out) = v;
            } else {
              out[0] = v.x;
              if (gcol + 1 < h) out[1] = v.y;
              if (gcol + 2 < h) out[2] = v.z;
              if (gcol + 3 < h) out[3] = v.w;
            }
          }
        }
        __syncwarp();
        if (hf + 1 < NP) tmem_wait16(rg2[(hf + 1) & 1]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[buf])) : "memory");
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, n_cols);
  }
}

// ---------------------------------------------------------------- warp-specialised split forms
// FP16 hi/lo split: A = A_hi + 2^-11 A_lo, B = B_hi + 2^-11 B_lo, and
//   A B ~ A_hi B_hi + 2^-11 (A_hi B_lo + A_lo B_hi)
// (the A_lo B_lo term is below FP32 rounding).  3xTF32 (TF32 = true) is the
// same with TF32 parts and no scaling (TF32 keeps the FP32 exponent range):
// A = A_hi + A_lo with A_hi = tf32(A), A_lo = tf32(A - A_hi).  A 16 KB operand
// block holds 128 rows x 64 FP16 or x 32 TF32 values.  One CTA per 128 rows
// and one column tile.  K runs in passes of `bp` blocks (the A_hi / A_lo
// blocks of a pass stay in shared memory while B_hi / B_lo stream through a
// 2-stage ring).  The tensor core's FP32 accumulation does not round to
// nearest: its error grows with the number of MMAs accumulated into one
// TMEM accumulator.  So the A_hi B_hi product of every K block goes to its own
// accumulator (three rotating 128-column TMEM buffers), which the epilogue
// warps drain into FP32 registers (round to nearest) as each block completes;
// the cross terms, 2^-11 smaller, share a fourth accumulator over all of K.
// Roles as in k_kernel_eval_tc_ta; the builders build a pass, then drain its
// blocks, and the drain of its last block (all MMAs before it complete) frees
// A for the next pass.
constexpr int kSpStages = 2;
constexpr int kSpMaxHalf = 4;  // blocks resident per pass

// NET = 3, the adjoint contraction Abar = c Gbar S^T of the differentiation
// form: A is Gbar[row][r] = gVW[row][r] + g_gamma[row] dgamma/dVWh[row][r]
// (K = h columns r), formed by the builders from these rows; the B image
// holds S[m][r] at (n = m - 1, k = r).
struct DenseA {
  const float* gVW;      // [rows][h] or null
  const float* VWh;      // [rows][h], the forward rows (sign of each entry)
  const float* g_gamma;  // [rows] or null
  int ca, cb, cr0;       // momentum grid: n_M = ca Q + cb, cr0 = -n_M/2 mod Q
};

// number of momentum indices M of the grid with M = r (mod Q)
__device__ __forceinline__ int grid_count_tc(int r, int Q, int a, int b, int r0) {
  int off = r - r0;
  if (off < 0) off += Q;
  return a + (off < b ? 1 : 0);
}

__device__ __forceinline__ float gbar_entry(const DenseA& g, int Q, int h, int row, int r) {
  if (r >= h) return 0.f;
  float v = g.gVW ? __ldg(g.gVW + (size_t)row * h + r) : 0.f;
  const float gg = g.g_gamma ? __ldg(g.g_gamma + row) : 0.f;
  if (gg != 0.f && r > 0) {
    const float w = __ldg(g.VWh + (size_t)row * h + r);
    const int dg = w > 0.f ? grid_count_tc(r, Q, g.ca, g.cb, g.cr0) : (w < 0.f ? -grid_count_tc(Q - r, Q, g.ca, g.cb, g.cr0) : 0);
    v = __fadd_rn(v, __fmul_rn(gg, (float)dg));
  }
  return v;
}
constexpr int kSpParts = 3;    // per-K-block accumulators (the cross-term accumulator is a fourth)

// blocks per pass: half of K for FP16 (one or two passes), 4 for TF32
__host__ __device__ constexpr int split_pass_blocks(int KB, bool tf32) {
  return tf32 ? 4 : ((KB + 1) / 2 < 4 ? (KB + 1) / 2 : 4);
}

__host__ __device__ constexpr size_t ws_split_smem_bytes(int KB, int h, bool tf32 = false) {
  return kSmemAlignPad + (size_t)2 * split_pass_blocks(KB, tf32) * kTileBytes + (size_t)kSpStages * 2 * kTileBytes +
         sizeof(float) * (size_t)((TM + 2 * h) > (kWsBuilders / 32) * kWsStageFloats
                                      ? (TM + 2 * h)
                                      : (kWsBuilders / 32) * kWsStageFloats);
}

template <bool TF32, int NET>
__global__ __launch_bounds__(kWsThreads, 1) void k_kernel_eval_tc_ws_split(
    const float* __restrict__ V, int n_x, int bc, int Q, const int* __restrict__ occ,
    const int* __restrict__ n_occ_dev, int n_occ_host, const void* __restrict__ img_hi_v,
    const void* __restrict__ img_lo_v, int KB, float c, float* __restrict__ VWh, unsigned int* __restrict__ flags,
    DenseA dense) {
  // FP16 x FP16 -> FP32 (format 0) or TF32 x TF32 -> FP32 (format 2)
  constexpr uint32_t idesc = idesc_f16(TF32 ? 2u : 0u);
  constexpr int KBLK = TF32 ? 32 : TK;   // K values per operand block
  constexpr int EPC = KBLK / 8;          // values per 16-byte chunk
  constexpr float kLoScale = TF32 ? 1.f : 0x1p-11f;
  const uint8_t* img_hi = static_cast<const uint8_t*>(img_hi_v);
  const uint8_t* img_lo = static_cast<const uint8_t*>(img_lo_v);
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = align_smem(smem_raw);
  const int bp = split_pass_blocks(KB, TF32);                 // blocks per pass
  uint8_t* sAh = smem;                                        // bp blocks of A_hi
  uint8_t* sAl = smem + (size_t)bp * kTileBytes;               // bp blocks of A_lo
  uint8_t* sB = smem + (size_t)2 * bp * kTileBytes;            // stages of (B_hi, B_lo)
  float* sV = reinterpret_cast<float*>(sB + (size_t)kSpStages * 2 * kTileBytes);  // shared with the staging
  __shared__ __align__(8) uint64_t a_ready[kSpMaxHalf];
  __shared__ __align__(8) uint64_t b_full[kSpStages], b_empty[kSpStages];
  __shared__ __align__(8) uint64_t acc_full[kSpParts], acc_empty[kSpParts], drain;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;

  const int n_rows = n_occ_dev ? *n_occ_dev : n_occ_host;
  const int row0 = blockIdx.x * TM;
  const int h = Q / 2;
  if (row0 >= n_rows) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nt = blockIdx.y;
  const int n_pass = (KB + bp - 1) / bp;
  const int n_tiles = KB;  // B tiles streamed: one per K block

  if (warp == 0) tmem_alloc(&tmem_slot, 512u);
  if (tid == 0) {
    for (int q = 0; q < kSpMaxHalf; ++q) mbar_init(&a_ready[q], kWsBuilders);
    for (int q = 0; q < kSpStages; ++q) {
      mbar_init(&b_full[q], 1);
      mbar_init(&b_empty[q], 1);
    }
    for (int q = 0; q < kSpParts; ++q) {
      mbar_init(&acc_full[q], 1);
      mbar_init(&acc_empty[q], kWsBuilders / 32);  // one arrival per epilogue warp
    }
    mbar_init(&drain, 1);
    fence_mbar_init();
    s_abort = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t acc_x = tmem + (uint32_t)(kSpParts * TN);  // cross terms; block buffers at tmem + TN b

  if (warp == kWsBuilders / 32 + 1) {
    // ---- B producer: tile kb of column tile nt, hi and lo, in K order
    if (lane == 0) {
      int issued = 0;
      for (int t = 0; t < n_tiles && !s_abort; ++t) {
        const int st = t % kSpStages;
        if (t >= kSpStages && !mbar_wait(&b_empty[st], (uint32_t)(((t / kSpStages) - 1) & 1))) {
          atomicOr(flags, WMC_FLAG_TIMEOUT);
          s_abort = 1;
          break;
        }
        uint8_t* dst = sB + (size_t)st * 2 * kTileBytes;
        const size_t off = ((size_t)nt * KB + t) * kTileBytes;  // bytes
        mbar_expect_tx(&b_full[st], 2 * kTileBytes);
        bulk_g2s(dst, img_hi + off, kTileBytes, &b_full[st]);
        bulk_g2s(dst + kTileBytes, img_lo + off, kTileBytes, &b_full[st]);
        issued = t + 1;
      }
      if (s_abort)
        for (int t = max(0, issued - kSpStages); t < issued; ++t)
          (void)mbar_wait(&b_full[t % kSpStages], (uint32_t)((t / kSpStages) & 1));
    }
  } else if (warp == kWsBuilders / 32) {
    // ---- MMA issuer
    if (lane == 0) {
      for (int pass = 0; pass < n_pass && !s_abort; ++pass) {
        const int kb0 = pass * bp, kb1 = min(KB, kb0 + bp);
        for (int kb = kb0; kb < kb1; ++kb) {
          const int kbl = kb - kb0, st = kb % kSpStages, buf = kb % kSpParts;
          if (!mbar_wait(&a_ready[kbl], (uint32_t)(pass & 1)) ||
              !mbar_wait(&b_full[st], (uint32_t)((kb / kSpStages) & 1)) ||
              (kb >= kSpParts && !mbar_wait(&acc_empty[buf], (uint32_t)(((kb / kSpParts) - 1) & 1)))) {
            atomicOr(flags, WMC_FLAG_TIMEOUT);
            s_abort = 1;
            break;
          }
          tc_fence_after();
          const uint32_t acc_m = tmem + (uint32_t)(buf * TN);
          const uint32_t ah = smem_u32(sAh + (size_t)kbl * kTileBytes), al = smem_u32(sAl + (size_t)kbl * kTileBytes);
          const uint32_t bh = smem_u32(sB + (size_t)st * 2 * kTileBytes), bl = bh + kTileBytes;
#pragma unroll
          for (int s4 = 0; s4 < TK / 16; ++s4) {
            const uint32_t o = s4 * kKStepBytes;
            const uint64_t dah = smem_desc(ah + o), dbh = smem_desc(bh + o);
            const bool first_m = s4 == 0;
            if (TF32) {
              mma_tf32(acc_m, dah, dbh, idesc, first_m ? 0u : 1u);
              mma_tf32(acc_x, dah, smem_desc(bl + o), idesc, (kb == 0 && s4 == 0) ? 0u : 1u);
              mma_tf32(acc_x, smem_desc(al + o), dbh, idesc, 1u);
            } else {
              mma_f16(acc_m, dah, dbh, idesc, first_m ? 0u : 1u);
              mma_f16(acc_x, dah, smem_desc(bl + o), idesc, (kb == 0 && s4 == 0) ? 0u : 1u);
              mma_f16(acc_x, smem_desc(al + o), dbh, idesc, 1u);
            }
          }
          mma_commit(&b_empty[st]);
          mma_commit(&acc_full[buf]);
        }
      }
      if (s_abort) {
        mma_commit(&drain);
        (void)mbar_wait(&drain, 0u);
      }
    }
  } else {
    // ---- A builders (warps 0-15): both passes, then the epilogue
    const int rc = tid & (TM - 1);
    const int rowc = row0 + rc;
    const bool validc = rowc < n_rows;
    const int cellc = validc ? (occ ? __ldg(occ + rowc) : rowc % n_x) : 0;
    const int potc = (occ || !validc) ? 0 : rowc / n_x;
    const int cell0 = occ ? __ldg(occ + row0) : row0 % n_x;
    const int pot0 = occ ? 0 : row0 / n_x;
    const bool contig = NET != 3 && builders_and(validc && cellc == cell0 + rc && potc == pot0);
    if (contig) {
      const float* V0 = V + (size_t)pot0 * n_x;
      constexpr int kU = 4;
      for (int q0 = tid; q0 < TM + 2 * h; q0 += kU * kWsBuilders) {
        float v[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int q = q0 + u * kWsBuilders;
          v[u] = q < TM + 2 * h ? potential_at(V0, n_x, bc, (long long)cell0 - h + q) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u)
          if (q0 + u * kWsBuilders < TM + 2 * h) sV[q0 + u * kWsBuilders] = v[u];
      }
      builders_sync();
    }
    const int rg = tid & 31, k8 = (tid >> 5) & 7, par = tid >> 8;
    int cell_d[4];
    bool valid_d[4];
    const float* V_d[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const int row = row0 + 4 * rg + d;
      valid_d[d] = row < n_rows;
      cell_d[d] = (contig || !valid_d[d]) ? 0 : (occ ? __ldg(occ + row) : row % n_x);
      V_d[d] = V + (size_t)((occ || !valid_d[d]) ? 0 : row / n_x) * n_x;
    }
    const bool fast = contig && (h & 3) == 0;
    // epilogue slice of warp w: TMEM lanes 32 (w % 4) .. + 31, columns 32 (w / 4) .. + 31
    const int quad = warp & 3, cq = warp >> 2;
    const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
    float sacc[32];  // sum over the K blocks drained so far of A_hi B_hi
#pragma unroll
    for (int q = 0; q < 32; ++q) sacc[q] = 0.f;
    bool drained_all = true;
    for (int pass = 0; pass < n_pass; ++pass) {
      const int kb0 = pass * bp, kb1 = min(KB, kb0 + bp), cnt = kb1 - kb0;
      for (int kbl = 1 - par; kbl < cnt; kbl += 2)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&a_ready[kbl])) : "memory");
#pragma unroll 1
      for (int kbl = par; kbl < cnt; kbl += 2) {
        const int kb = kb0 + kbl;
        const int m0 = kb * KBLK + k8 * EPC + 1;
        float dv[4][EPC];
        if (NET == 1 && fast && m0 + EPC - 1 <= h - 1) {
          // P[j] = V at offset m0 - 1 + j right of row 4 rg, N[j] = V at offset m0 + EPC - 1 - j left of it
          constexpr int NW = EPC + 4;
          float P[NW], N[NW];
          const float* pp = sV + 4 * rg + h + m0 - 1;
          const float* pn = sV + 4 * rg + h - m0 - (EPC - 1);
#pragma unroll
          for (int q = 0; q < NW / 4; ++q) {
            const float4 a = *reinterpret_cast<const float4*>(pp + 4 * q);
            const float4 b = *reinterpret_cast<const float4*>(pn + 4 * q);
            P[4 * q] = a.x, P[4 * q + 1] = a.y, P[4 * q + 2] = a.z, P[4 * q + 3] = a.w;
            N[4 * q] = b.x, N[4 * q + 1] = b.y, N[4 * q + 2] = b.z, N[4 * q + 3] = b.w;
          }
#pragma unroll
          for (int d = 0; d < 4; ++d)
#pragma unroll
            for (int e = 0; e < EPC; ++e) dv[d][e] = __fsub_rn(P[d + e + 1], N[d - e + EPC - 1]);
        } else if (NET == 3) {
          const int r0 = m0 - 1;
          if ((h & 3) == 0 && EPC == 4 && r0 + 3 < h) {
            // four consecutive columns of each row: one 16-byte load per operand
            float4 gv[4], wv[4];
            float gg[4];
#pragma unroll
            for (int d = 0; d < 4; ++d) {
              const size_t o = (size_t)(row0 + 4 * rg + d) * h + r0;
              gv[d] = (valid_d[d] && dense.gVW) ? __ldg(reinterpret_cast<const float4*>(dense.gVW + o))
                                                : make_float4(0.f, 0.f, 0.f, 0.f);
              gg[d] = (valid_d[d] && dense.g_gamma) ? __ldg(dense.g_gamma + row0 + 4 * rg + d) : 0.f;
              wv[d] = (valid_d[d] && gg[d] != 0.f) ? __ldg(reinterpret_cast<const float4*>(dense.VWh + o))
                                                   : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int d = 0; d < 4; ++d) {
              const float g4[4] = {gv[d].x, gv[d].y, gv[d].z, gv[d].w};
              const float w4[4] = {wv[d].x, wv[d].y, wv[d].z, wv[d].w};
#pragma unroll
              for (int e = 0; e < EPC; ++e) {
                const int r = r0 + e;
                float v = g4[e];
                if (gg[d] != 0.f && r > 0) {
                  const int dg = w4[e] > 0.f ? grid_count_tc(r, Q, dense.ca, dense.cb, dense.cr0)
                                             : (w4[e] < 0.f ? -grid_count_tc(Q - r, Q, dense.ca, dense.cb, dense.cr0) : 0);
                  v = __fadd_rn(v, __fmul_rn(gg[d], (float)dg));
                }
                dv[d][e] = valid_d[d] ? v : 0.f;
              }
            }
          } else {
#pragma unroll
            for (int d = 0; d < 4; ++d)
#pragma unroll
              for (int e = 0; e < EPC; ++e)
                dv[d][e] = valid_d[d] ? gbar_entry(dense, Q, h, row0 + 4 * rg + d, m0 - 1 + e) : 0.f;
          }
        } else {
#pragma unroll
          for (int d = 0; d < 4; ++d)
#pragma unroll
            for (int e = 0; e < EPC; ++e) {
              const int kk = m0 - 1 + e;
              dv[d][e] = 0.f;
              if (contig) dv[d][e] = a_entry_window<NET == 3 ? 1 : NET>(sV + 4 * rg + d, h, cell0 + 4 * rg + d, kk);
              else if (valid_d[d]) dv[d][e] = a_term<NET == 3 ? 1 : NET>(V_d[d], n_x, bc, h, cell_d[d], kk);
            }
        }
        uint4 wh[4], wl[4];
#pragma unroll
        for (int d = 0; d < 4; ++d) {
          uint32_t hw[4], lw[4];
          if (TF32) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              hw[e] = to_tf32(dv[d][e]);
              lw[e] = to_tf32(__fsub_rn(dv[d][e], __uint_as_float(hw[e])));
            }
          } else {
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
              const uint16_t h0 = to_bits(dv[d][e], WMC_FP16), h1 = to_bits(dv[d][e + 1], WMC_FP16);
              const uint16_t l0 = to_bits(__fmul_rn(__fsub_rn(dv[d][e], from_bits(h0, WMC_FP16)), 2048.f), WMC_FP16);
              const uint16_t l1 =
                  to_bits(__fmul_rn(__fsub_rn(dv[d][e + 1], from_bits(h1, WMC_FP16)), 2048.f), WMC_FP16);
              hw[e / 2] = (uint32_t)h0 | ((uint32_t)h1 << 16);
              lw[e / 2] = (uint32_t)l0 | ((uint32_t)l1 << 16);
            }
          }
          wh[d] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          wl[d] = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
        uint8_t* bh = sAh + (size_t)kbl * kTileBytes;
        uint8_t* bl = sAl + (size_t)kbl * kTileBytes;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int x = (i + (rg >> 1)) & 3;
          const uint32_t off = core_offset(4 * rg + x, k8 * 8);
          *reinterpret_cast<uint4*>(bh + off) = x == 0 ? wh[0] : x == 1 ? wh[1] : x == 2 ? wh[2] : wh[3];
          *reinterpret_cast<uint4*>(bl + off) = x == 0 ? wl[0] : x == 1 ? wl[1] : x == 2 ? wl[2] : wl[3];
        }
        fence_proxy_async_smem();
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&a_ready[kbl])) : "memory");
      }
      // drain the pass's K blocks in order; after the last one every MMA that
      // reads this pass's A has completed, so the next pass may overwrite it
      for (int kb = kb0; kb < kb1 && drained_all; ++kb) {
        const int buf = kb % kSpParts;
        int okw = 1;
        if (lane == 0) okw = !s_abort && mbar_wait(&acc_full[buf], (uint32_t)((kb / kSpParts) & 1));
        if (__shfl_sync(0xffffffffu, okw, 0) == 0) {  // warp-uniform: the TMEM loads are warp-collective
          if (lane == 0) atomicOr(flags, WMC_FLAG_TIMEOUT);
          s_abort = 1;
          drained_all = false;
          break;
        }
        tc_fence_after();
        uint32_t r0[16], r1[16];
        const uint32_t ta = tmem + (uint32_t)(buf * TN) + lane_base + (uint32_t)(cq * 32);
        tmem_ld16_issue(ta, r0);
        tmem_ld16_issue(ta + 16u, r1);
        tmem_wait16(r0);
        tmem_wait16(r1);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          sacc[q] = __fadd_rn(sacc[q], __uint_as_float(r0[q]));
          sacc[16 + q] = __fadd_rn(sacc[16 + q], __uint_as_float(r1[q]));
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0)
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[buf])) : "memory");
      }
      if (!drained_all) break;
    }
    // epilogue: v = c (sum of the block products + 2^-11 x cross)
    float* stg = sV + warp * kWsStageFloats;
    const bool vec_ok = (h & 3) == 0 && (reinterpret_cast<uintptr_t>(VWh) & 15) == 0;
    if (drained_all) {
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        const int cc = cq * 32 + hf * 16;
        const int col0 = nt * TN + cc;
        float a[16], x[16];
        tmem_ld16(acc_x + lane_base + (uint32_t)cc, x);
#pragma unroll
        for (int q = 0; q < 16; ++q) a[q] = __fmul_rn(c, __fadd_rn(sacc[hf * 16 + q], __fmul_rn(x[q], kLoScale)));
#pragma unroll
        for (int g = 0; g < 4; ++g)
          *reinterpret_cast<float4*>(stg + lane * 16 + 4 * (g ^ ((lane >> 1) & 3))) =
              make_float4(a[4 * g], a[4 * g + 1], a[4 * g + 2], a[4 * g + 3]);
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int rr = 8 * i + (lane >> 2), g = lane & 3;
          const float4 v = *reinterpret_cast<const float4*>(stg + rr * 16 + 4 * (g ^ ((rr >> 1) & 3)));
          const int grow = row0 + quad * 32 + rr, gcol = col0 + 4 * g;
          if (grow < n_rows && gcol < h) {
            float* out = VWh + (size_t)grow * h + gcol;
            if (vec_ok) {
              *reinterpret_cast<float4*>(out) = v;
            } else {
              out[0] = v.x;
              if (gcol + 1 < h) out[1] = v.y;
              if (gcol + 2 < h) out[2] = v.z;
              if (gcol + 3 < h) out[3] = v.w;
            }
          }
        }
        __syncwarp();
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 512u);
  }
}

// ---------------------------------------------------------------- host side
struct TcImages {
  int KB, NT, KB32, KB2;     // 16-bit K blocks (64 values), column tiles, TF32 K blocks (32 values), N = 2 K blocks
  int KBa;                   // the adjoint's TF32 K blocks (K = h), Q <= 256 only (else 0)
  size_t bytes_per_image;    // NT * KB * kTileBytes (BF16, FP16 hi, FP16 lo)
  size_t bytes_per_image32;  // NT * KB32 * kTileBytes (TF32 hi, TF32 lo)
  size_t bytes_per_image2;   // NT * KB2 * kTileBytes (N = 2 network: BF16, FP16 hi, FP16 lo)
  size_t bytes_per_imagea;   // NT * KBa * kTileBytes (adjoint, TF32 hi, TF32 lo)
};

static int g_h(const wmc_params& p) { return p.Q / 2; }

static TcImages tc_geometry(const wmc_params& p) {
  TcImages g;
  const int h = p.Q / 2;
  g.KB = (h - 1 + TK - 1) / TK;
  if (g.KB < 1) g.KB = 1;
  g.NT = (h + TN - 1) / TN;
  g.KB32 = (h - 1 + 31) / 32;
  if (g.KB32 < 1) g.KB32 = 1;
  g.KB2 = (h + TK - 1) / TK;  // the N = 2 network's K = h pair offsets
  g.bytes_per_image = (size_t)g.NT * g.KB * kTileBytes;
  g.bytes_per_image32 = (size_t)g.NT * g.KB32 * kTileBytes;
  g.bytes_per_image2 = (size_t)g.NT * g.KB2 * kTileBytes;
  g.KBa = h <= kAdjMaxH ? (h + 31) / 32 : 0;
  g.bytes_per_imagea = (size_t)g.NT * g.KBa * kTileBytes;
  return g;
}

size_t tc_images_bytes(const wmc_params& p) {
  const TcImages g = tc_geometry(p);
  return 3 * g.bytes_per_image + 2 * g.bytes_per_image32 + 3 * g.bytes_per_image2 + 2 * g.bytes_per_imagea;
}

static const uint8_t* adjoint_images(const void* images, const TcImages& g) {
  return static_cast<const uint8_t*>(images) + 3 * g.bytes_per_image + 2 * g.bytes_per_image32 +
         3 * g.bytes_per_image2;
}

cudaError_t launch_init_tc_images(const wmc_params& p, void* images, cudaStream_t s) {
  const TcImages g = tc_geometry(p);
  uint16_t* base = static_cast<uint16_t*>(images);
  const size_t n16 = g.bytes_per_image / 2;
  k_init_tc_images<<<256, 256, 0, s>>>(p.Q, g.KB, g.NT, base, base + n16, base + 2 * n16, 1);
  uint32_t* b32 = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(images) + 3 * g.bytes_per_image);
  k_init_tc_images32<<<256, 256, 0, s>>>(p.Q, g.KB32, g.NT, b32, b32 + g.bytes_per_image32 / 4, 0);
  uint16_t* b2 = reinterpret_cast<uint16_t*>(static_cast<uint8_t*>(images) + 3 * g.bytes_per_image +
                                             2 * g.bytes_per_image32);
  const size_t n2 = g.bytes_per_image2 / 2;
  k_init_tc_images<<<256, 256, 0, s>>>(p.Q, g.KB2, g.NT, b2, b2 + n2, b2 + 2 * n2, 2);
  if (g.KBa) {
    uint32_t* ba = reinterpret_cast<uint32_t*>(const_cast<uint8_t*>(adjoint_images(images, g)));
    k_init_tc_images32<<<256, 256, 0, s>>>(p.Q, g.KBa, g.NT, ba, ba + g.bytes_per_imagea / 4, 1);
  }
  return cudaGetLastError();
}

// Abar = c Gbar S^T on the 3xTF32 split kernel (NET = 3), rows = n_pot n_x
// implicit rows; Q <= 256.
cudaError_t launch_adjoint_abar_tc(const wmc_params& p, int rows, const float* VWh, const float* gVW,
                                   const float* g_gamma, const void* images, float* Abar, unsigned int* flags,
                                   cudaStream_t s) {
  const TcImages g = tc_geometry(p);
  if (!g.KBa) return cudaErrorNotSupported;
  if (rows <= 0) return cudaSuccess;
  const uint8_t* ba = adjoint_images(images, g);
  DenseA d;
  d.gVW = gVW;
  d.VWh = VWh;
  d.g_gamma = g_gamma;
  d.ca = p.n_M / p.Q;
  d.cb = p.n_M - d.ca * p.Q;
  d.cr0 = ((-(p.n_M / 2)) % p.Q + p.Q) % p.Q;
  const float c = (float)(-2.0 / (kHbarEVs * (double)p.Q));
  const size_t sm = ws_split_smem_bytes(g.KBa, g_h(p), true);
  const dim3 grid((rows + TM - 1) / TM, g.NT);
  cudaError_t e = raise_smem_limit(reinterpret_cast<const void*>(k_kernel_eval_tc_ws_split<true, 3>), sm);
  if (e != cudaSuccess) return e;
  k_kernel_eval_tc_ws_split<true, 3><<<grid, kWsThreads, sm, s>>>(nullptr, rows, 0, p.Q, nullptr, nullptr, rows, ba,
                                                                  ba + g.bytes_per_imagea, g.KBa, c, Abar, flags, d);
  return cudaGetLastError();
}

// The form behind a requested precision: WMC_FP32 takes the 3xTF32 split
// kernel (N = 1 network, where its shared memory holds the window) for
// Q > 256, and for Q >= 128 when the rows fill a wave of 128-row tiles on
// every SM (rows > 0: the row entry points; measured 2.4x faster than the
// CUDA cores at Q = 256 over 262144 rows, error 1.6e-7 against 2.2e-7);
// else the CUDA-core form.  WMC_FP32_SIMT is always the CUDA-core form.  The
// result is the internal code: WMC_FP32 then always means the CUDA cores.
int resolve_precision(const wmc_params& p, int prec, int net, long long rows) {
  if (prec == WMC_FP32_SIMT) return WMC_FP32;
  if (prec != WMC_FP32 || net != 1) return prec;
  if (p.Q <= 256 && !(p.Q >= 128 && rows >= (long long)TM * num_sms())) return prec;
  const TcImages g = tc_geometry(p);
  return ws_split_smem_bytes(g.KB32, g_h(p), true) <= 226 * 1024 ? WMC_TF32X3 : WMC_FP32;
}

// The N = 2 network (net = 2) runs on the warp-specialised BF16 / FP16 and
// FP16-split kernels with its own operand images and A builder; other forms
// return cudaErrorNotSupported for it.
template <int NET>
static cudaError_t launch_tc_net(const wmc_params& p, int prec, const float* V, const int* occ, const int* n_occ_dev,
                                 int n_occ_host, int max_rows, const uint16_t* base, int KB, const TcImages& g,
                                 float* VWh, unsigned int* flags, cudaStream_t s);

cudaError_t launch_kernel_eval_tc(const wmc_params& p, int prec, const float* V, const int* occ, const int* n_occ_dev,
                                  int n_occ_host, int max_rows, const void* images, float* VWh, unsigned int* flags,
                                  cudaStream_t s, int net) {
  if (max_rows <= 0) return cudaSuccess;
  const TcImages g = tc_geometry(p);
  if (net == 2) {
    const uint16_t* b2 = reinterpret_cast<const uint16_t*>(static_cast<const uint8_t*>(images) +
                                                           3 * g.bytes_per_image + 2 * g.bytes_per_image32);
    return launch_tc_net<2>(p, prec, V, occ, n_occ_dev, n_occ_host, max_rows, b2, g.KB2, g, VWh, flags, s);
  }
  const uint16_t* base = static_cast<const uint16_t*>(images);
  if (prec == WMC_BF16 || prec == WMC_FP16 || prec == WMC_FP16_SPLIT) {
    const cudaError_t e = launch_tc_net<1>(p, prec, V, occ, n_occ_dev, n_occ_host, max_rows, base, g.KB, g, VWh,
                                           flags, s);
    if (e != cudaErrorNotSupported) return e;
  }
  const size_t n16 = g.bytes_per_image / 2;
  const float c = (float)(-2.0 / (kHbarEVs * (double)p.Q));
  dim3 grid((max_rows + TM - 1) / TM, g.NT);
  if (prec == WMC_BF16) {
    const size_t sm = tc_smem_bytes(false, g_h(p));
    raise_smem_limit(reinterpret_cast<const void*>(k_kernel_eval_tc<WMC_BF16>), sm);
    k_kernel_eval_tc<WMC_BF16><<<grid, 128, sm, s>>>(V, p.n_x, p.bc_potential, p.Q, occ, n_occ_dev, n_occ_host,
                                                     base, nullptr, g.KB, c, VWh, flags);
  } else if (prec == WMC_FP16) {
    const size_t sm = tc_smem_bytes(false, g_h(p));
    raise_smem_limit(reinterpret_cast<const void*>(k_kernel_eval_tc<WMC_FP16>), sm);
    k_kernel_eval_tc<WMC_FP16><<<grid, 128, sm, s>>>(V, p.n_x, p.bc_potential, p.Q, occ, n_occ_dev, n_occ_host,
                                                     base + n16, nullptr, g.KB, c, VWh, flags);
  } else if (prec == WMC_TF32X3 && ws_split_smem_bytes(g.KB32, g_h(p), true) <= 226 * 1024) {
    const size_t sm = ws_split_smem_bytes(g.KB32, g_h(p), true);
    const uint8_t* b32 = reinterpret_cast<const uint8_t*>(images) + 3 * g.bytes_per_image;
    raise_smem_limit(reinterpret_cast<const void*>(k_kernel_eval_tc_ws_split<true, 1>), sm);
    k_kernel_eval_tc_ws_split<true, 1><<<grid, kWsThreads, sm, s>>>(V, p.n_x, p.bc_potential, p.Q, occ, n_occ_dev,
                                                                 n_occ_host, b32, b32 + g.bytes_per_image32,
                                                                 g.KB32, c, VWh, flags, DenseA{});
  } else if (prec == WMC_FP16_SPLIT) {
    const size_t sm = tc_smem_bytes(true, g_h(p));
    raise_smem_limit(reinterpret_cast<const void*>(k_kernel_eval_tc<WMC_FP16_SPLIT>), sm);
    k_kernel_eval_tc<WMC_FP16_SPLIT><<<grid, 128, sm, s>>>(V, p.n_x, p.bc_potential, p.Q, occ, n_occ_dev,
                                                           n_occ_host, base + n16, base + 2 * n16, g.KB, c, VWh,
                                                           flags);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int NET>
static cudaError_t launch_tc_net(const wmc_params& p, int prec, const float* V, const int* occ, const int* n_occ_dev,
                                 int n_occ_host, int max_rows, const uint16_t* base, int KB, const TcImages& g,
                                 float* VWh, unsigned int* flags, cudaStream_t s) {
  const size_t n16 = (size_t)g.NT * KB * kTileBytes / 2;
  const float c = (float)(-2.0 / (kHbarEVs * (double)p.Q));
  const int row_tiles = (max_rows + TM - 1) / TM;
  if ((prec == WMC_BF16 || prec == WMC_FP16) && KB <= kTaMaxKB && ta_smem_bytes(g_h(p)) <= 226 * 1024) {
    // A in tensor memory.  The 128-column tiles are split over grid.y by the
    // factor that minimises waves x per-CTA work, with the fixed part of a CTA
    // (set-up and building A) counted as three column tiles.
    const uint16_t* img = prec == WMC_BF16 ? base : base + n16;
    const long long sms = num_sms();
    int n_split = 1;
    long long best = -1;
    for (int ns = 1; ns <= g.NT; ns *= 2) {
      const long long waves = ((long long)row_tiles * ns + sms - 1) / sms;
      const long long cost = waves * (3 + (long long)((g.NT + ns - 1) / ns));
      if (best < 0 || cost < best) {
        best = cost;
        n_split = ns;
      }
    }
    const size_t sm = ta_smem_bytes(g_h(p));
    const void* fn = prec == WMC_BF16 ? reinterpret_cast<const void*>(k_kernel_eval_tc_ta<WMC_BF16, NET>)
                                      : reinterpret_cast<const void*>(k_kernel_eval_tc_ta<WMC_FP16, NET>);
    const cudaError_t e = raise_smem_limit(fn, sm);
    if (e != cudaSuccess) return e;
    const dim3 grid(row_tiles, n_split);
    if (prec == WMC_BF16)
      k_kernel_eval_tc_ta<WMC_BF16, NET><<<grid, kWsThreads, sm, s>>>(V, p.n_x, p.bc_potential, p.Q, occ, n_occ_dev,
                                                                      n_occ_host, img, KB, g.NT, n_split, c, VWh,
                                                                      flags);
    else
      k_kernel_eval_tc_ta<WMC_FP16, NET><<<grid, kWsThreads, sm, s>>>(V, p.n_x, p.bc_potential, p.Q, occ, n_occ_dev,
                                                                      n_occ_host, img, KB, g.NT, n_split, c, VWh,
                                                                      flags);
    return cudaGetLastError();
  }
  if (prec == WMC_FP16_SPLIT && ws_split_smem_bytes(KB, g_h(p)) <= 226 * 1024) {
    const size_t sm = ws_split_smem_bytes(KB, g_h(p));
    const dim3 grid(row_tiles, g.NT);
    raise_smem_limit(reinterpret_cast<const void*>(k_kernel_eval_tc_ws_split<false, NET>), sm);
    k_kernel_eval_tc_ws_split<false, NET><<<grid, kWsThreads, sm, s>>>(V, p.n_x, p.bc_potential, p.Q, occ,
                                                                       n_occ_dev, n_occ_host, base + n16,
                                                                       base + 2 * n16, KB, c, VWh, flags, DenseA{});
    return cudaGetLastError();
  }
  return cudaErrorNotSupported;
}

}  // namespace wmc
