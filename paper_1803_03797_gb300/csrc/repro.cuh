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
// 2^(32k - 1074); a block value adds three 32-bit digits, which a warp
// combines over its lanes into sums below 2^37 before adding, so a limb absorbs
// 2^26 warp additions -- one per 1024 grid points: 2^36 points per dot --
// before it could overflow; larger grids are rejected on the host.
#pragma once

#include "common.cuh"

namespace lap5 {

constexpr int kExactRows = 16;   // block height (kExactLimbs, kExactSlots: common.cuh)

// Whole warp: add every lane's v exactly to L.  Lanes whose lowest digit
// falls within four limbs of the warp's lowest combine their digits first --
// integer sums of 16-bit halves, exact -- so the warp issues at most six
// atomics for them instead of three per lane; other lanes add their own digits.
// Non-finite values set *bad.
__device__ __forceinline__ void exact_add_warp(unsigned long long* L, unsigned* bad, double v) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const unsigned ex = (unsigned)(bits >> 52) & 0x7ffu;
  const bool nonfinite = ex == 0x7ffu;
  if (__any_sync(full, nonfinite) && lane == 0) atomicOr(bad, 1u);
  const bool use = !nonfinite && v != 0.0;
  unsigned long long m = bits & 0xfffffffffffffull;
  int o = 0;  // weight of m's lowest bit: 2^(o - 1074)
  if (ex != 0) {
    m |= 1ull << 52;
    o = (int)ex - 1;
  }
  const int k = o >> 5, sh = o & 31;
  const unsigned long long lo = m << sh;
  const unsigned long long hi = sh ? (m >> (64 - sh)) : 0ull;
  const unsigned d0 = (unsigned)(lo & 0xffffffffull), d1 = (unsigned)(lo >> 32), d2 = (unsigned)hi;
  const bool neg = (bits >> 63) != 0ull;
  const int kmin = __reduce_min_sync(full, use ? k : 0x7fffffff);
  if (kmin == 0x7fffffff) return;  // no lane holds a nonzero value
  const int off = k - kmin;
  const bool near = use && off < 4;
  if (use && !near) {  // two's complement digits (the limbs are signed)
    const unsigned long long s0 = neg ? 0ull - d0 : d0, s1 = neg ? 0ull - d1 : d1, s2 = neg ? 0ull - d2 : d2;
    if (s0) atomicAdd(&L[k], s0);
    if (s1) atomicAdd(&L[k + 1], s1);
    if (s2) atomicAdd(&L[k + 2], s2);
  }
  long long mine = 0;
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    const int q = p - off;
    const unsigned dig = !near ? 0u : (q == 0) ? d0 : (q == 1) ? d1 : (q == 2) ? d2 : 0u;
    const int l16 = (int)(dig & 0xffffu), h16 = (int)(dig >> 16);
    const int sl = __reduce_add_sync(full, neg ? -l16 : l16);
    const int sh16 = __reduce_add_sync(full, neg ? -h16 : h16);
    if (lane == p) mine = (long long)sl + (long long)sh16 * 65536ll;
  }
  if (lane < 6 && mine != 0 && kmin + lane < kExactLimbs) atomicAdd(&L[kmin + lane], (unsigned long long)mine);
}

// Whole warp: lowest and highest nonzero limb of L (lo = kExactLimbs if none).
__device__ __forceinline__ void exact_range(const long long* L, int& lo, int& hi) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned b0 = __ballot_sync(full, L[lane] != 0);
  const unsigned b1 = __ballot_sync(full, L[lane + 32] != 0);
  const unsigned b2 = __ballot_sync(full, lane + 64 < kExactLimbs && L[lane + 64] != 0);
  lo = b0 ? __ffs(b0) - 1 : b1 ? 32 + __ffs(b1) - 1 : b2 ? 64 + __ffs(b2) - 1 : kExactLimbs;
  hi = b2 ? 64 + 31 - __clz(b2) : b1 ? 32 + 31 - __clz(b1) : b0 ? 31 - __clz(b0) : -1;
}

// Round the exact total to binary64 (nearest, ties to even).  L holds the
// limbs (shared memory), nonzero only within [lo, hi]; normalised in place.
// One thread.
__device__ inline double exact_round(long long* L, bool bad, int lo, int hi) {
  if (bad) return __longlong_as_double(0x7ff8000000000000ll);
  if (lo >= kExactLimbs) return 0.0;
  // digits in [0, 2^32) from lo upwards; a negative total borrows up to the
  // top limb, which then holds its sign.  Returns the highest limb touched.
  auto normalise = [&](int from, int until) -> int {
    long long c = 0;
    int k = from;
    for (; k + 1 < kExactLimbs; ++k) {
      const long long t = L[k] + c;
      c = t >> 32;  // arithmetic shift: floor division
      L[k] = t - c * (1ll << 32);
      if (k >= until && c == 0) return k;
    }
    L[kExactLimbs - 1] += c;
    return kExactLimbs - 1;
  };
  int top = normalise(lo, hi);
  const bool neg = L[top] < 0;
  if (neg) {
    for (int k = lo; k <= top; ++k) L[k] = -L[k];
    top = normalise(lo, top);
  }
  int h = top;
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
            if (L) exact_add_warp(L, bad, c);
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
  {
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int k = warp; k < NV; k += nwarps) {
      long long* Lk = reinterpret_cast<long long*>(tm.xs + k * kExactLimbs);
      int lo, hi;
      exact_range(Lk, lo, hi);
      if ((threadIdx.x & 31) == 0) {
        const bool bad = __ldcg(&ctl->xbad[e][k]) != 0u;
        red[32 * kMaxVals + k] = exact_round(Lk, bad, lo, hi);
      }
      __syncwarp();
    }
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
