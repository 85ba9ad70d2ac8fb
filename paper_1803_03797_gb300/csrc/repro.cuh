// repro.cuh -- reproducible dot products: a value that does not depend on how
// the grid is split over CTAs, warps and lanes, on the lane vector width or on
// the ring.
//
// The paper accumulates in fixed point because floating-point addition is not
// associative and would tie the result to one order of operations (Sec. III;
// the dot product itself is a multiplier-adder tree, Sec. II-C-1).  Here:
//   1. blocks of 2 columns x 16 rows aligned at column 2c and row 16t; points
//      outside the grid have a = b = 0;
//   2. row value of a block: fma(a1, b1, a0*b0), a0*b0 rounded first;
//   3. block value: a fixed pairwise tree over the block's 16 row values
//      (rows 2m and 2m+1, then pairs of those, ...);
//   4. (a, b): the exact sum of all block values, rounded once to nearest
//      (ties to even); an exact zero is +0; a non-finite block value gives NaN.
// Step 3 runs in registers while a warp marches its unit (units start at
// multiples of 16 rows, so a block never straddles two warps); step 4 adds each
// block value exactly into a fixed-point accumulator -- the paper's fixed-point
// accumulation, widened to the whole binary64 range -- first one per CTA in
// shared memory, then one per solve in global memory, and rounds the total.
//
// The accumulator: kExactLimbs signed 64-bit limbs, limb k weighing
// 2^(32k - 1074); each block value adds three 32-bit digits, so a limb absorbs
// 2^31 additions before it could overflow (2^36 grid points per dot).
#pragma once

#include "common.cuh"

namespace lap5 {

constexpr int kExactRows = 16;   // block height (kExactLimbs, kExactSlots: common.cuh)

// Add v exactly to the accumulator L (shared or global; atomics, so any
// number of threads may add at once).  Non-finite v sets *bad.
__device__ __forceinline__ void exact_add(unsigned long long* L, unsigned* bad, double v) {
  if (v == 0.0) return;
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const unsigned ex = (unsigned)(bits >> 52) & 0x7ffu;
  if (ex == 0x7ffu) {
    atomicOr(bad, 1u);
    return;
  }
  unsigned long long m = bits & 0xfffffffffffffull;
  int o = 0;  // weight of m's lowest bit: 2^(o - 1074)
  if (ex != 0) {
    m |= 1ull << 52;
    o = (int)ex - 1;
  }
  const int k = o >> 5, sh = o & 31;
  const unsigned long long lo = m << sh;
  const unsigned long long hi = sh ? (m >> (64 - sh)) : 0ull;
  unsigned long long d0 = lo & 0xffffffffull, d1 = lo >> 32, d2 = hi;
  if (bits >> 63) {  // subtract: two's complement digits (the limbs are signed)
    d0 = 0ull - d0;
    d1 = 0ull - d1;
    d2 = 0ull - d2;
  }
  if (d0) atomicAdd(&L[k], d0);
  if (d1) atomicAdd(&L[k + 1], d1);
  if (d2) atomicAdd(&L[k + 2], d2);
}

// Round the exact total to binary64 (nearest, ties to even).  L holds the
// limbs (shared memory) and is normalised in place; one thread.
__device__ inline double exact_round(long long* L, bool bad) {
  if (bad) return __longlong_as_double(0x7ff8000000000000ll);
  int lo = 0, hi = kExactLimbs - 1;
  while (lo < kExactLimbs && L[lo] == 0) ++lo;
  if (lo == kExactLimbs) return 0.0;
  while (L[hi] == 0) --hi;
  // digits in [0, 2^32), the top limb carries the sign; carries stop a few
  // limbs above the highest nonzero one
  auto normalise = [&]() {
    long long c = 0;
    for (int k = lo; k + 1 < kExactLimbs; ++k) {
      const long long t = L[k] + c;
      c = t >> 32;  // arithmetic shift: floor division
      L[k] = t - c * (1ll << 32);
      if (k >= hi && c == 0) break;
    }
    if (c != 0) L[kExactLimbs - 1] += c;
  };
  normalise();
  int top = kExactLimbs - 1;
  while (top > lo && L[top] == 0) --top;
  const bool neg = L[top] < 0;
  if (neg) {
    for (int k = lo; k <= top; ++k) L[k] = -L[k];
    hi = top;
    normalise();
  }
  int h = kExactLimbs - 1;
  while (h >= lo && L[h] == 0) --h;
  if (h < lo) return 0.0;
  auto D = [&](int k) -> unsigned long long { return k >= lo ? (unsigned long long)L[k] : 0ull; };
  double r;
  if (h <= 1 && ((D(1) << 32) | D(0)) < (1ull << 53)) {
    r = ldexp((double)((D(1) << 32) | D(0)), -1074);  // exact
  } else {
    const unsigned long long w = (D(h) << 32) | D(h - 1);
    const int lz = __clzll(w);  // < 32: the top digit is nonzero
    const unsigned long long d2 = D(h - 2);
    const unsigned long long t64 = lz ? ((w << lz) | (d2 >> (32 - lz))) : w;
    bool sticky = (lz ? (d2 & ((1ull << (32 - lz)) - 1ull)) : d2) != 0ull;
    for (int k = h - 3; k >= lo && !sticky; --k) sticky = L[k] != 0;
    int pos = 32 * h + 31 - lz;  // bit index of the leading one (weight 2^(pos - 1074))
    unsigned long long q = t64 >> 11;
    const unsigned long long rem = t64 & 0x7ffull;
    if (rem > 0x400ull || (rem == 0x400ull && (sticky || (q & 1ull)))) ++q;
    if (q == (1ull << 53)) {
      q >>= 1;
      ++pos;
    }
    r = ldexp((double)q, pos - 52 - 1074);  // exact (normal range) or infinite
  }
  return neg ? -r : r;
}

// Steps 2 and 3 for one lane of a binary64 warp strip (two columns a lane):
// the block tree of the lane's column pair, fed one row at a time in the
// unit's march order; a completed block is added to the CTA accumulator.
struct AccExact {
  static constexpr bool kExact = true;
  unsigned long long* L = nullptr;  // CTA accumulator of this dot (nullptr: discard)
  unsigned* bad = nullptr;
  int ny = 0;
  bool rev = false;
  int n = 0;  // rows fed into the current block
  double p0 = 0.0, p1 = 0.0, p2 = 0.0, p3 = 0.0;

  __device__ __forceinline__ void feed(double v) {
    double c = v;
    if (n & 1) {
      c = p0 + c;
      if (n & 2) {
        c = p1 + c;
        if (n & 4) {
          c = p2 + c;
          if (n & 8) {
            c = p3 + c;
            if (L) exact_add(L, bad, c);
          } else {
            p3 = c;
          }
        } else {
          p2 = c;
        }
      } else {
        p1 = c;
      }
    } else {
      p0 = c;
    }
    n = (n + 1) & (kExactRows - 1);
  }
  // Rows of the grid's last, partial block that do not exist: +0, fed before
  // the block's rows when marching down and after them when marching up, so
  // that the tree pairs the same rows either way.
  __device__ __forceinline__ void pad() {
    const int m = ny % kExactRows;
    for (int k = m; k < kExactRows; ++k) feed(0.0);
  }
  // Row j of the lane: a[k], b[k] at the lane's columns x, x+1 (ncols = nx - x).
  template <int V>
  __device__ __forceinline__ void row(int j, const double (&a)[V], const double (&b)[V], int ncols) {
    static_assert(V == 2, "exact dot products take two columns a lane");
    const double a0 = ncols > 0 ? a[0] : 0.0, b0 = ncols > 0 ? b[0] : 0.0;
    const double a1 = ncols > 1 ? a[1] : 0.0, b1 = ncols > 1 ? b[1] : 0.0;
    const double v = __fma_rn(a1, b1, __dmul_rn(a0, b0));
    const bool last = (j == ny - 1) && (ny % kExactRows) != 0;
    if (last && rev) pad();
    feed(v);
    if (last && !rev) pad();
  }
};

template <int V>
__device__ __forceinline__ void acc_dot(AccExact& acc, int j, const double (&a)[V], const double (&b)[V], int ncols) {
  acc.template row<V>(j, a, b, ncols);
}

template <class Acc> struct AccTraits { static constexpr bool kExact = false; };
template <> struct AccTraits<AccExact> { static constexpr bool kExact = true; };

// An accumulator for dot slot `slot` of the next reduction (slot < 0: an
// exact accumulator that discards), for a pass marching down (rev) or up.
template <class Acc, class Team>
__device__ __forceinline__ Acc make_acc(Team& tm, int slot, int ny, bool rev) {
  Acc a{};
  if constexpr (AccTraits<Acc>::kExact) {
    a.L = slot >= 0 ? tm.xs + slot * kExactLimbs : nullptr;
    a.bad = slot >= 0 ? tm.xsb + slot : nullptr;
    a.ny = ny;
    a.rev = rev;
  } else {
    (void)tm; (void)slot; (void)ny; (void)rev;
  }
  return a;
}

// Exact reduction of the NV dot products accumulated in the CTAs' shared
// accumulators (slots 0..NV-1): every CTA adds its accumulators into the
// solve's global accumulator of this reduction, the grid barrier, then every
// CTA rounds the totals (identical in every CTA).  Buffers rotate over three
// exact reductions; CTA 0 clears the next one before it arrives: its last
// readers finished two exact reductions ago, and its next writers start after
// this barrier.
template <int NV>
__device__ __forceinline__ bool grid_reduce_exact(GridTeam& tm, double (&out)[NV], double* red) {
  static_assert(NV <= kExactSlots, "too many exact dot products");
  const int e = (int)(tm.xepoch % 3u);
  Ctl* ctl = tm.ctl;
  __syncthreads();  // every block value of this CTA is in its accumulators
  for (int t = threadIdx.x; t < NV * kExactLimbs; t += blockDim.x) {
    const unsigned long long v = tm.xs[t];
    if (v) atomicAdd(&ctl->xacc[e][0][0] + t, v);
    tm.xs[t] = 0ull;
  }
  if (threadIdx.x < NV) {
    if (tm.xsb[threadIdx.x]) atomicOr(&ctl->xbad[e][threadIdx.x], 1u);
    tm.xsb[threadIdx.x] = 0u;
  }
  if (blockIdx.x == 0) {
    const int en = (e + 1) % 3;
    for (int t = threadIdx.x; t < kExactSlots * kExactLimbs; t += blockDim.x) (&ctl->xacc[en][0][0])[t] = 0ull;
    if (threadIdx.x < kExactSlots) ctl->xbad[en][threadIdx.x] = 0u;
  }
  ++tm.xepoch;
  double v[1] = {0.0}, o[1];
  if (!grid_reduce<1>(ctl, tm.epoch, v, o, red, tm.timeout_ns)) return false;
  // the totals, read past L1 (other SMs' atomics landed in L2); the CTA's own
  // accumulators are zero again and serve as scratch
  for (int t = threadIdx.x; t < NV * kExactLimbs; t += blockDim.x)
    tm.xs[t] = __ldcg(&ctl->xacc[e][0][0] + t);
  __syncthreads();
  if (threadIdx.x < NV) {
    const bool bad = __ldcg(&ctl->xbad[e][threadIdx.x]) != 0u;
    red[32 * kMaxVals + threadIdx.x] =
        exact_round(reinterpret_cast<long long*>(tm.xs + threadIdx.x * kExactLimbs), bad);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NV * kExactLimbs; t += blockDim.x) tm.xs[t] = 0ull;
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = red[32 * kMaxVals + k];
  __syncthreads();
  return true;
}

// Drop what the CTA's exact accumulators hold (a pass whose dot products are
// not needed after all).  Call after a barrier that every warp of the CTA has
// passed since its last addition.
template <class Acc, class Team>
__device__ __forceinline__ void acc_discard(Team& tm) {
  if constexpr (AccTraits<Acc>::kExact) {
    for (int t = threadIdx.x; t < kExactSlots * kExactLimbs; t += blockDim.x) tm.xs[t] = 0ull;
    if (threadIdx.x < kExactSlots) tm.xsb[threadIdx.x] = 0u;
    __syncthreads();
  } else {
    (void)tm;
  }
}

// Reduce NV accumulators of one kind: plain values through the team's
// reduction, exact ones through grid_reduce_exact.
template <int NV, class Team, class Acc>
__device__ __forceinline__ bool acc_reduce(Team& tm, Acc* const (&accs)[NV], double (&out)[NV], double* red) {
  if constexpr (AccTraits<Acc>::kExact) {
    return grid_reduce_exact<NV>(tm, out, red);
  } else {
    double v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = accs[k]->value();
    return tm.template reduce<NV>(v, out, red);
  }
}

}  // namespace lap5
