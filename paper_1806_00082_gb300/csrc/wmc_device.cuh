// Device helpers shared by the libwmc kernels (single simulation and batched).
#pragma once

#include <stdint.h>

#include "wmc_internal.cuh"

namespace wmc {

// Entry (kk, r) of the sine matrix of the N = 1 network (the folded window sum
// of Eq. wigner-1d-discrete): sin(2 pi ((kk+1) r mod Q) / Q) for kk < h-1,
// r < h (term m = kk + 1, half-period column r), zero elsewhere.  Every
// kernel and operand image takes its sine values from here.
__device__ __forceinline__ float sine_entry_n1(int Q, int kk, int r) {
  const int h = Q / 2;
  if (kk >= h - 1 || r >= h) return 0.f;
  const long long t = ((long long)(kk + 1) * r) % Q;
  return __double2float_rn(sinpi(2.0 * (double)t / (double)Q));
}

// Entry (u, r) of the matrix of the N = 2 barycentric network in its folded
// form (Eq. kernel_ML with N = 2): cos(pi r / Q) sin(pi ((2u+1) r mod 2Q) / Q)
// for u < h, r < h (pair offset u, half-period column r), zero elsewhere; the
// product is formed in FP64 and rounded once.
__device__ __forceinline__ float sine_entry_n2(int Q, int u, int r) {
  const int h = Q / 2;
  if (u >= h || r >= h) return 0.f;
  const long long t = ((long long)(2 * u + 1) * r) % (2ll * Q);
  return __double2float_rn(cospi((double)r / (double)Q) * sinpi((double)t / (double)Q));
}

__device__ __forceinline__ float pot(const float* __restrict__ V, int n_x, int bc, long long l) {
  if (l >= 0 && l < n_x) return __ldg(V + l);
  if (!bc) return 0.f;
  return __ldg(V + (l < 0 ? 0 : n_x - 1));
}

// Term idx of the contraction's A operand for cell i of potential V: the N = 1
// network's difference V(i + m) - V(i - m), m = idx + 1 (zero from idx = h - 1
// on), or the N = 2 network's signed pair sum at offset u = idx:
// V(i+u) + V(i+u+1) if i + u is even, else -(V(i-u-1) + V(i-u)) (zero from
// idx = h on); the pair at u and its mirror at -u-1 have opposite sines and
// exactly one of them starts at an even cell.
template <int NET>
__device__ __forceinline__ float a_term(const float* __restrict__ V, int n_x, int bc, int h, long long i, int idx) {
  if (NET == 1) {
    const int m = idx + 1;
    return m <= h - 1 ? __fsub_rn(pot(V, n_x, bc, i + m), pot(V, n_x, bc, i - m)) : 0.f;
  }
  const int u = idx;
  if (u > h - 1) return 0.f;
  return ((i + u) & 1) == 0 ? __fadd_rn(pot(V, n_x, bc, i + u), pot(V, n_x, bc, i + u + 1))
                            : -__fadd_rn(pot(V, n_x, bc, i - u - 1), pot(V, n_x, bc, i - u));
}

// Error-free transformation of a + b (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum_acc(float& s, float& e, float p) {
  const float sn = __fadd_rn(s, p);
  const float bp = __fsub_rn(sn, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(sn, bp)), __fsub_rn(p, bp));
  s = sn;
  e = __fadd_rn(e, err);
}

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

__device__ __forceinline__ float positive_part_smem(const float* v, int Q, int r) {
  const int h = Q / 2;
  float x = 0.f;
  if (r != 0 && r != h) x = r < h ? v[r] : -v[Q - r];
  return x > 0.f ? x : 0.f;
}

// total 2^-s as a double: the conversion of total rounds to nearest, the
// power of two (built from its bits) scales exactly; two FP64 operations,
// where the library ldexp costs many on the narrow FP64 pipe.
__device__ __forceinline__ double scaled_total(long long total, int s) {
  if (s > -1023 && s < 1023) return __dmul_rn((double)total, __longlong_as_double((long long)(1023 - s) << 52));
  return ldexp((double)total, -s);
}

// The fixed-point CDF of one row held in a warp: lane l takes the contiguous
// columns k in [l E, (l+1) E), E = ceil(n_M / 32), so a row needs one warp
// reduction (maximum), one warp scan of the lane totals and E sequential
// integer additions per lane; lanes write contiguous runs of the row-major CDF.
// Column k has momentum residue (r0 + k) mod Q (r0 = -n_M/2 mod Q); xres(rr)
// returns max(V_W, 0) at residue rr, stepped incrementally along a lane's run.
// zero_rows: also write the all-zero CDF of a row without positive entries
// (the simulation step never reads it: such a row has gamma = 0, so no pair is
// drawn from it).
// coarse (optional): the row's coarse CDF, lane l's inclusive sum at coarse[l]
// (the CDF at the last column of block l), written for rows with positive
// entries.
template <class XRes>
__device__ __forceinline__ void warp_row_cdf(XRes xres, int Q, int r0, int n_M, int log2_nM, int lane,
                                             long long* __restrict__ out, double& gamma_out, int& scale_out,
                                             long long& total_out, bool zero_rows = true,
                                             long long* __restrict__ coarse = nullptr) {
  const int E = (n_M + 31) >> 5;
  const int k0 = min(lane * E, n_M), k1 = min(k0 + E, n_M);
  const int rr0 = (r0 + k0) % Q;
  uint32_t mx = 0u;
  for (int k = k0, rr = rr0; k < k1; ++k) {
    mx = max(mx, __float_as_uint(xres(rr)));
    if (++rr == Q) rr = 0;
  }
  mx = __reduce_max_sync(0xffffffffu, mx);
  if (mx == 0u) {
    if (out && zero_rows)
      for (int k = k0; k < k1; ++k) out[k] = 0;
    gamma_out = 0.0;
    scale_out = 0;
    total_out = 0;
    return;
  }
  const int s = 61 - log2_nM - floor_log2_pos(__uint_as_float(mx));
  long long local = 0;
  for (int k = k0, rr = rr0; k < k1; ++k) {
    local += quantise(xres(rr), s);
    if (++rr == Q) rr = 0;
  }
  long long incl = local;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const long long u = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += u;
  }
  const long long total = __shfl_sync(0xffffffffu, incl, 31);
  if (coarse) coarse[lane] = incl;
  if (out) {
    long long run = incl - local;
    for (int k = k0, rr = rr0; k < k1; ++k) {
      run += quantise(xres(rr), s);
      out[k] = run;
      if (++rr == Q) rr = 0;
    }
  }
  gamma_out = scaled_total(total, s);
  scale_out = s;
  total_out = total;
}

// gthr = ceil(fl64(gamma dt) 2^32), flagging gamma dt >= 1.
__device__ __forceinline__ unsigned long long event_threshold(double g, double dt, unsigned int* flags) {
  const double gd = __dmul_rn(g, dt);
  if (gd >= 1.0) {
    atomicOr(flags, WMC_FLAG_RATE);
    return 1ull << 32;
  }
  return (unsigned long long)ceil(gd * 4294967296.0);
}

// Loads the signed counts of cell i into s_n and the exclusive prefix of |n|
// into s_pre[0..n_M] (s_pre[n_M] = survivors of the cell), by one warp: 32
// columns at a time (lane l takes column k0 + l, so the loads coalesce and the
// shared-memory stores hit distinct banks), a warp scan per chunk and a carry.
__device__ __forceinline__ void warp_row_prefix(const int32_t* __restrict__ hist, int i, int n_M, int* s_n,
                                                int* s_pre, int lane) {
  const int32_t* row = hist + (size_t)i * n_M;
  int carry = 0;
  for (int k0 = 0; k0 < n_M; k0 += 32) {
    const int k = k0 + lane;
    const int n = k < n_M ? __ldg(row + k) : 0;
    const int v = n < 0 ? -n : n;
    int incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += u;
    }
    if (k < n_M) {
      s_n[k] = n;
      s_pre[k] = carry + incl - v;
    }
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) s_pre[n_M] = carry;
}

// Cell i needs its kernel row this step: occupied, or a neighbour drifts into
// it (reach bits: 1 occupied, 2 has a rightward momentum, 4 a leftward one).
__device__ __forceinline__ int cell_needs_kernel(const unsigned char* reach, int i, int n_x) {
  return (reach[i] & 1) || (i > 0 && (reach[i - 1] & 2)) || (i + 1 < n_x && (reach[i + 1] & 4));
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

// Drift direction of column k from its thresholds: +1, -1, or 0 (never moves).
__device__ __forceinline__ int drift_dir(uint32_t lo, uint32_t hi) { return hi != 0xffffffffu ? 1 : (lo ? -1 : 0); }

// Index of p' for the 53-bit uniform integer U2 in a fixed-point CDF row c of
// n_M columns: target = floor(U2 Qtot / 2^53), Qtot = c[n_M - 1], and the
// smallest k with c[k] > target (always exists, since target < Qtot).
__device__ __forceinline__ int sample_cdf_row(const long long* __restrict__ c, int n_M, unsigned long long U2) {
  const unsigned long long Qtot = (unsigned long long)__ldg(c + n_M - 1);
  const long long target = (long long)((__umul64hi(U2, Qtot) << 11) | ((U2 * Qtot) >> 53));
  int lo = 0, hi = n_M - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(c + mid) > target) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// Index of p' for the 53-bit uniform integer U2 from a coarse CDF: cc[l] is the
// CDF at the last column of lane block l (E columns each, E = ceil(n_M / 32))
// and the block's own columns are re-quantised from the kernel row v (scale
// s), so the result is the smallest k with C[k] > floor(U2 C[n_M - 1] / 2^53)
// exactly as with the full CDF.  Column k has residue (r0 + k) mod Q.  Loads
// go out in small independent groups: the four segment ends of the 32 block
// sums, the eight sums of one segment, then the block's columns eight at a
// time.
__device__ __forceinline__ int sample_coarse_row(const float* __restrict__ v, const long long* __restrict__ cc,
                                                 int s, int Q, int r0, int n_M, unsigned long long U2) {
  const long long e0 = __ldg(cc + 7), e1 = __ldg(cc + 15), e2 = __ldg(cc + 23), e3 = __ldg(cc + 31);
  const unsigned long long Qtot = (unsigned long long)e3;
  const long long target = (long long)((__umul64hi(U2, Qtot) << 11) | ((U2 * Qtot) >> 53));
  const int seg = (e0 <= target) + (e1 <= target) + (e2 <= target);  // e3 > target always
  const longlong2* cs = reinterpret_cast<const longlong2*>(cc + 8 * seg);
  long long c8[8];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const longlong2 pr = __ldg(cs + j);
    c8[2 * j] = pr.x;
    c8[2 * j + 1] = pr.y;
  }
  int blk = 8 * seg;
  long long run = seg == 0 ? 0ll : (seg == 1 ? e0 : (seg == 2 ? e1 : e2));
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const bool below = c8[j] <= target;
    blk += below;
    run = below ? c8[j] : run;  // the CDF before block blk
  }
  const int E = (n_M + kCdfBlocks - 1) / kCdfBlocks;
  const int k0 = min(blk * E, n_M), k1 = min(k0 + E, n_M);
  const int h = Q / 2;
  int rr = (r0 + k0) % Q;
  for (int kb = k0; kb < k1; kb += 8) {
    float x[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      int r = rr + e;
      r = r >= Q ? r - Q : r;
      float val = 0.f;
      if (kb + e < k1 && r != 0 && r != h) val = r < h ? __ldg(v + r) : -__ldg(v + (Q - r));
      x[e] = val > 0.f ? val : 0.f;
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      run += quantise(x[e], s);
      if (kb + e < k1 && run > target) return kb + e;
    }
    rr += 8;
    rr = rr >= Q ? rr - Q : rr;
  }
  return k1 - 1;  // not reached: block blk's sum exceeds the target
}

// The same draw with sequential loads and few registers (for the rare calls
// from inside the particle-step kernel).
__device__ __forceinline__ int sample_coarse_row_seq(const float* __restrict__ v, const long long* __restrict__ cc,
                                                     int s, int Q, int r0, int n_M, unsigned long long U2) {
  const unsigned long long Qtot = (unsigned long long)__ldg(cc + kCdfBlocks - 1);
  const long long target = (long long)((__umul64hi(U2, Qtot) << 11) | ((U2 * Qtot) >> 53));
  int lo = 0, hi = kCdfBlocks - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(cc + mid) > target) hi = mid; else lo = mid + 1;
  }
  const int E = (n_M + kCdfBlocks - 1) / kCdfBlocks;
  const int k0 = min(lo * E, n_M), k1 = min(k0 + E, n_M);
  long long run = lo ? __ldg(cc + lo - 1) : 0ll;
  int rr = (r0 + k0) % Q;
  for (int k = k0; k < k1; ++k) {
    run += quantise(positive_part(v, Q, rr), s);
    if (run > target) return k;
    if (++rr == Q) rr = 0;
  }
  return k1 - 1;
}

// Smallest j in [0, 2^24] with fl32(j 2^-24 + d) >= edge (2^24 if none); the
// predicate is monotone in j because rounding is.
__device__ __forceinline__ int first_offset_reaching(float d, float edge) {
  int lo = 0, hi = 1 << 24;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__fadd_rn((float)mid * 0x1p-24f, d) >= edge) hi = mid; else lo = mid + 1;
  }
  return lo;
}

}  // namespace wmc
