// Internal declarations shared by the libwmc translation units: workspace
// layout, device header, Philox4x32-10 and launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include "wmc.h"

namespace wmc {

// Host-side NVTX range for one phase of a call (visible to profilers that
// record NVTX; a no-op otherwise).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr double kHbarEVs = 6.582119569e-16;  // hbar [eV s]
constexpr double kHbarJs = 1.054571817e-34;   // hbar [J s]
constexpr double kPi = 3.14159265358979323846;

// Philox counter word 2 of each draw.  A particle with number id takes word
// id % 4 of counter (id / 4, step, purpose, sim) for its offset (REPOS) and its
// pair-creation uniform (GEN); a created pair draws p' from words 0, 1 of
// (id, step, PICK, sim).
constexpr uint32_t kPurposeGen = 1u;
constexpr uint32_t kPurposeRepos = 2u;
constexpr uint32_t kPurposePick = 3u;

// Step work decomposition: the survivors of cell i (ids R[i] .. R[i] + T[i] - 1)
// are cut into work items on a grid of kChunk ids aligned to A = R[i] rounded
// down to a multiple of 4: item c of cell i holds the ids in
// [A + c kChunk, A + (c+1) kChunk) that belong to the cell, so every Philox
// call (four consecutive ids) stays within one item.  A cell has
// ceil((T[i] + 3) / kChunk) items (the last may be empty).  A warp of the
// particle-step kernel takes one item at a time, each lane a quad-aligned run
// of at most kChunk / 32 consecutive ids.
constexpr int kStepThreads = 256;
constexpr int kStepWarps = kStepThreads / 32;
constexpr int kChunk = 2048;
constexpr int kMaxStepBlocks = 8192;
constexpr long long kMaxItemsBase = 1ll << 20;   // item descriptors: 2^32 / kChunk + n_x
// Lane blocks of the coarse momentum CDF: a row's n_M columns are cut into 32
// blocks of E = ceil(n_M / 32) consecutive columns (block l is [l E, (l+1) E)).
constexpr int kCdfBlocks = 32;
// Cells per block of the plan's scan.
constexpr int kPlanCells = 1024;

constexpr unsigned kMagic = 0x574d4331u;  // "WMC1": set by wmc_init

// Lives at offset 0 of the workspace.
struct DevHeader {
  unsigned long long population;      // survivors enumerated by the last plan
  unsigned long long particle_steps;  // cumulative
  unsigned long long pairs;
  unsigned long long absorbed;
  long long absorbed_signed;
  unsigned long long dropped;
  long long dropped_signed;
  int n_items;
  int n_occ;
  unsigned int flags;
  unsigned int step;    // device step counter (wmc_run)
  unsigned int magic;
  unsigned int item_ticket;  // next work item of the running step launch
  unsigned int blocks_done;  // step blocks finished (the last one resets both)
  unsigned int rows_by_cell; // 1: the kernel stage wrote its rows at the cell index, 0: at the occupied-list index
  unsigned int pair_count;   // pair events queued by the particle-step kernel (reset by the pair kernel)
  unsigned int pairs_done;   // pair-kernel blocks finished (the last one resets the queue and the ticket)
  unsigned int plan_epoch;   // launches of the plan so far (tags its blocks' published prefixes)
  unsigned int plan_ticket;  // logical block index of the running plan launch (reset by its last block)
  unsigned int chunk;        // ids per work item of the current plan (0: kChunk)
  unsigned long long id_base;  // number of the first survivor (a sub-domain numbers after the cells before it)
  unsigned int chunk_next;   // the plan's choice for the next step (the pair kernel makes it current)
  unsigned int pad1;
};

// Totals of a run of cells in the plan's scan: survivors (64 bits), work
// items, needed cells, and whether a cell held 2^31 survivors or more.
struct PlanSums {
  unsigned long long T;
  int I, N;
  int big;
  int pad;
};

// One block of the plan's scan publishes its own totals (agg) and then the
// totals of every cell up to its last (inc); tag = epoch << 2 | state, state
// 1 = agg valid, 2 = inc valid too, written after the values.
struct PlanStatus {
  PlanSums agg, inc;
  unsigned int tag;
  unsigned int pad[3];
};

// Byte offsets of the workspace regions (all 256-aligned).
struct Layout {
  size_t header, T, R, IP, reach, occ, row_map, VWh, ccdf, scale, gamma, gthr, thr_cell, D, xlo, xhi, items, pairs, B,
      B2, tc, plan, dft, total;
  long long max_items;
  unsigned pair_cap;  // entries of the pair queue
  int h;     // Q / 2
  int Kp;    // contraction length h - 1 padded to a multiple of 32
  int Np;    // output columns h padded to a multiple of 64
  int Kp2;   // contraction length h of the N = 2 network padded to a multiple of 32
};

bool params_ok(const wmc_params* p);
Layout layout(const wmc_params& p);

// Device pointers of one workspace.
struct View {
  DevHeader* hdr;
  unsigned long long* T;   // [n_x] survivors per cell
  unsigned long long* R;   // [n_x + 1] first id of each cell (exclusive prefix of T)
  int* IP;                 // [n_x + 1] first work item of each cell
  unsigned char* reach;    // [n_x] bit0 occupied, bit1 some drift right, bit2 some drift left
  int* occ;                // [n_x] occupied-cell list (ascending)
  int* row_map;            // [n_x] cell -> row of occ, or -1
  float* VWh;              // [n_x][h] kernel half-period rows, by occ row
  long long* ccdf;         // [n_x][kCdfBlocks] coarse fixed-point CDF by occ row (inclusive block sums)
  int* scale;              // [n_x] fixed-point scale s of each row
  double* gamma;           // [n_x] gamma by occ row
  unsigned long long* gthr;// [n_x] event threshold by occ row: word < gthr <=> word 2^-32 < gamma dt
  unsigned long long* thr_cell;  // [n_x] the same by cell (0 for cells without a kernel row)
  float* D;                // [n_M] drift per step in cells
  uint32_t* xlo;           // [n_M] offset word w crosses left iff w < xlo[k]
  uint32_t* xhi;           // [n_M] ... crosses right iff w > xhi[k]
  int2* items;             // [max_items] work items (cell, chunk)
  uint4* pairs;            // [pair_cap] pair events (id, cell, column, sign < 0) queued by the step
  float* B;                // [Kp][Np] sine matrix S[m][r], m = kk + 1
  float* B2;               // [Kp2][Np] folded matrix of the N = 2 network, pair offset u
  void* tc;                // tensor-core operand images of S (BF16, FP16 hi, FP16 lo)
  PlanStatus* plan;        // [ceil(n_x / kPlanCells)] published prefixes of the plan's blocks
  double* dft;             // [2 Q] cos and sin of the Q phases (sliding-window evaluation)
};
View view(const wmc_params& p, void* ws);

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, SC'11: ten rounds of two 32x32 -> 64-bit
// multiplications (0xD2511F53, 0xCD9E8D57) with the word permutation of the
// four-word variant, and a Weyl key schedule (0x9E3779B9, 0xBB67AE85).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
  }
  return c;
}

// Two Philox4x32-10 evaluations under one key and one key schedule.
__device__ __forceinline__ void philox4x32_10_x2(uint4& a, uint4& b, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * a.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * a.z;
    const unsigned long long q0 = (unsigned long long)0xD2511F53u * b.x;
    const unsigned long long q1 = (unsigned long long)0xCD9E8D57u * b.z;
    a = make_uint4((uint32_t)(p1 >> 32) ^ a.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ a.w ^ k1, (uint32_t)p0);
    b = make_uint4((uint32_t)(q1 >> 32) ^ b.y ^ k0, (uint32_t)q1, (uint32_t)(q0 >> 32) ^ b.w ^ k1, (uint32_t)q0);
  }
}

// The round keys of Philox4x32-10 under key (k0, k1): rk[2 r], rk[2 r + 1] =
// k0 + r W0, k1 + r W1 (r = 0..9), the Weyl sequence of the key schedule.
struct PhiloxKeys {
  uint32_t rk[20];
};

__host__ __device__ inline PhiloxKeys philox_keys(uint32_t k0, uint32_t k1) {
  PhiloxKeys K;
  for (int r = 0; r < 10; ++r) {
    K.rk[2 * r] = k0 + (uint32_t)r * 0x9E3779B9u;
    K.rk[2 * r + 1] = k1 + (uint32_t)r * 0xBB67AE85u;
  }
  return K;
}

// The same two evaluations with the round keys read from K: inside a kernel
// whose parameters hold K, the keys are constant operands of the XORs and the
// key schedule costs no instructions.
__device__ __forceinline__ void philox4x32_10_x2k(uint4& a, uint4& b, const PhiloxKeys& K) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * a.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * a.z;
    const unsigned long long q0 = (unsigned long long)0xD2511F53u * b.x;
    const unsigned long long q1 = (unsigned long long)0xCD9E8D57u * b.z;
    a = make_uint4((uint32_t)(p1 >> 32) ^ a.y ^ K.rk[2 * r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ a.w ^ K.rk[2 * r + 1],
                   (uint32_t)p0);
    b = make_uint4((uint32_t)(q1 >> 32) ^ b.y ^ K.rk[2 * r], (uint32_t)q1, (uint32_t)(q0 >> 32) ^ b.w ^ K.rk[2 * r + 1],
                   (uint32_t)q0);
  }
}

__device__ __forceinline__ uint4 philox4x32_10k(uint4 c, const PhiloxKeys& K) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ K.rk[2 * r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ K.rk[2 * r + 1],
                   (uint32_t)p0);
  }
  return c;
}

// Work items of a cell holding t survivors (an upper bound when its first id
// is not a multiple of 4; surplus items are empty).
__host__ __device__ __forceinline__ int items_of_cell(unsigned long long t, unsigned int chunk = kChunk) {
  return t ? (int)((t + 3 + chunk - 1) / chunk) : 0;
}

// Ids per work item: the header's current choice (kChunk until a step has
// chosen); a power of two in [kMinChunk, kChunk].
constexpr unsigned int kMinChunk = 512;
__device__ __forceinline__ unsigned int work_chunk(const DevHeader* hdr) {
  const unsigned int c = *(const volatile unsigned int*)&hdr->chunk;
  return c ? c : (unsigned int)kChunk;
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_init_tables(const wmc_params& p, const View& v, cudaStream_t s);
cudaError_t launch_plan(const wmc_params& p, const View& v, const int32_t* hist, int64_t* rho, int advance_step,
                        cudaStream_t s, int32_t* zero_out = nullptr);
// the two halves of launch_plan: the per-cell scan, and the single-block plan
// (clear_thr: also zero the event thresholds of every cell)
cudaError_t launch_rows(const wmc_params& p, const View& v, const int32_t* hist, int64_t* rho, cudaStream_t s,
                        int32_t* zero_out);
cudaError_t launch_plan_scan(const wmc_params& p, const View& v, int advance_step, int clear_thr, cudaStream_t s);
int step_grid(int n_M);
// (net 1: the N = 1 network with B = the sine matrix; net 2: the N = 2
// network with B = its folded matrix B2)
cudaError_t launch_kernel_eval(const wmc_params& p, const float* V, const int* occ, const int* n_occ_dev,
                               int n_occ_host, int max_rows, const float* B, float* VWh, cudaStream_t s,
                               int net = 1);
// Fused kernel row + fixed-point CDF for small windows (Q/2 <= 128); the CDF
// outputs may all be null (kernel rows only).
bool small_window(const wmc_params& p);
cudaError_t launch_kernel_rows_small(const wmc_params& p, const float* V, const int* occ, const int* n_occ_dev,
                                     int n_occ_host, int max_rows, const float* B, float* VWh, long long* ccdf,
                                     int* scale, double* gamma, unsigned long long* gthr,
                                     unsigned long long* thr_cell, unsigned int* flags, cudaStream_t s,
                                     const unsigned char* reach = nullptr, DevHeader* hdr = nullptr, int net = 1);
cudaError_t launch_gather_table(const wmc_params& p, const float* table, const int* occ, const int* n_occ_dev,
                                int max_rows, float* VWh, cudaStream_t s);
// Tensor-core contraction (BF16, FP16, FP16 hi/lo split).
size_t tc_images_bytes(const wmc_params& p);
cudaError_t launch_init_tc_images(const wmc_params& p, void* images, cudaStream_t s);
cudaError_t launch_kernel_eval_tc(const wmc_params& p, int prec, const float* V, const int* occ, const int* n_occ_dev,
                                  int n_occ_host, int max_rows, const void* images, float* VWh, unsigned int* flags,
                                  cudaStream_t s, int net = 1);
// CDF of rows: row-major cdf[row][n_M] and/or the coarse form ccdf[row][kCdfBlocks];
// cdf/ccdf/scale/gthr/thr_cell/flags may be null.
cudaError_t launch_cdf(const wmc_params& p, const float* VWh, const int* n_rows_dev, int n_rows_host,
                       int max_rows, long long* cdf, double* gamma, int* scale, unsigned long long* gthr,
                       const int* occ, unsigned long long* thr_cell, unsigned int* flags, cudaStream_t s,
                       DevHeader* hdr = nullptr, long long* ccdf = nullptr);
cudaError_t launch_step(const wmc_params& p, const View& v, const int32_t* hist_in, uint32_t t, int t_from_device,
                        int32_t* hist_out, cudaStream_t s);
cudaError_t launch_materialize(const wmc_params& p, const View& v, const int32_t* hist, uint32_t t, int32_t* cell,
                               float* f, int16_t* M, int8_t* sign, long long capacity, cudaStream_t s);
cudaError_t launch_density(const wmc_params& p, const int32_t* hist, int64_t* rho, cudaStream_t s);
// Every cell's kernel row by the FP64 sliding window (CS: 2 Q doubles of scratch).
int resolve_precision(const wmc_params& p, int prec, int net, long long rows = 0);
// The differentiation form's window limit (Q <= 256) and its Abar contraction
// on the tensor cores.
constexpr int kAdjMaxH = 128;
cudaError_t launch_adjoint_abar_tc(const wmc_params& p, int rows, const float* VWh, const float* gVW,
                                   const float* g_gamma, const void* images, float* Abar, unsigned int* flags,
                                   cudaStream_t s);
cudaError_t launch_kernel_dft(const wmc_params& p, const float* V, double* CS, float* VWh, cudaStream_t s);
cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, long long n, uint32_t* out,
                          cudaStream_t s);
cudaError_t launch_philox_throughput(uint32_t k0, uint32_t k1, int pairs_per_thread, uint32_t* out, long long n_threads,
                                     cudaStream_t s);

int num_sms();
// Raises a kernel's dynamic shared-memory limit (kept per kernel, device and
// context; the runtime is called only when the limit has to grow).
cudaError_t raise_smem_limit(const void* func, size_t bytes);
// Optional CUDA events around the particle-step kernel (wmc_step_timing): records
// the begin (end = false) or end event of the current device on s, as an
// event-record node when s is being captured.  No-op while timing is off.
cudaError_t step_timing_record(cudaStream_t s, bool end);
// Whether step timing is on (part of the key of the cached step graphs).
int step_timing_on();
// Caches the step kernel's launch shape for this device (call outside graph capture).
void prepare_step(const wmc_params& p);

}  // namespace wmc
