// ring.cuh -- per-warp shared-memory row ring filled by 1D bulk asynchronous
// copies (cp.async.bulk, the TMA engine's non-tensor form) and completed on
// mbarriers.
//
// A warp streams the rows of its unit in march order.  Lane 0 issues, S rows
// ahead, one bulk copy per streamed vector and row into a ring slot; the whole
// warp waits on the slot's mbarrier (bounded by %globaltimer), reads its 16-byte
// lane vectors from shared memory, and releases the slot for the row S ahead.
// Stencil operands are copied with the 16-byte chunks that hold the strip's
// halo columns, so a unit needs no scalar halo loads and no registers for rows
// in flight.  Bulk copies need 16-byte aligned rows and 16-byte multiples,
// which the solver's row layout (ld a multiple of the lane vector, rows 16-byte
// aligned) guarantees.
#pragma once

#include "common.cuh"

namespace lap5 {

constexpr int kRingMaxVecs = 6;
constexpr int kRingMaxSlots = 8;
constexpr uint32_t kSuspendHintNs = 64;  // upper bound on one try_wait suspension

enum { RV_HALO = 1, RV_ALWAYS = 2 };  // stencil operand; also needed on the unit's halo rows

struct RingVec {
  const unsigned char* base;  // element (0, 0)
  int ld;                     // row pitch in elements
  int es;                     // element bytes
  int flags;
};

// Ring geometry chosen on the host: slots per warp and bytes per slot.
struct RingGeom {
  int S;           // slots per warp (0 = ring disabled)
  int slot_bytes;  // >= the largest slot any pass of the kernel needs
  int warp_bytes;  // shared bytes per warp: barriers + slots
};

__host__ __device__ inline int ring_seg_bytes(int V, int es, bool halo) { return 32 * V * es + (halo ? 32 : 0); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

struct WarpRing {
  uint32_t bars;       // shared address of S mbarriers (8 bytes each)
  uint32_t slots;      // shared address of slot 0
  unsigned char* slots_ptr;
  int S, slot_bytes;
  unsigned q;          // sequence number of the next row to produce / consume
  unsigned q_issued;   // rows produced so far (lane 0)
  int pslot;           // slot of the next produce (lane 0)
  int cslot;           // slot of the next wait
  uint32_t cpar;       // phase parity the next wait expects
  bool failed;
  long long timeout_ns;
  int* err;
  int* abort_flag;

  __device__ __forceinline__ void init(unsigned char* warp_smem, const RingGeom& g, long long to, int* err_word,
                                       int* abort_word) {
    S = g.S;
    slot_bytes = g.slot_bytes;
    bars = smem_u32(warp_smem);
    slots_ptr = warp_smem + 128;  // 8 barriers padded to 128 bytes
    slots = smem_u32(slots_ptr);
    q = 0;
    q_issued = 0;
    pslot = 0;
    cslot = 0;
    cpar = 0;
    failed = false;
    timeout_ns = to;
    err = err_word;
    abort_flag = abort_word;
    if ((threadIdx.x & 31) == 0) {
      for (int s = 0; s < S; ++s)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bars + 8u * s) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
  }

  // Per-unit copy plan: for each vector the byte range of the strip (with its
  // halo chunks) inside a row, where it lands in the slot, and the bytes an
  // interior / halo row brings.  Computed once per unit so that producing a
  // row costs one row-offset multiply-add and one copy instruction per vector.
  template <int V, int K>
  struct Plan {
    const unsigned char* src[K];  // base + first byte of the strip's range (row 0)
    size_t row_bytes[K];          // ld * es
    uint32_t dst[K];              // shared address offset inside a slot
    int nb[K];                    // bytes per row (0: not streamed)
    bool always[K];               // also on the unit's halo rows
    uint32_t tx_interior, tx_halo;
  };

  template <int V, int K>
  __device__ __forceinline__ static void plan(Plan<V, K>& P, int xs, const RingVec (&v)[K], const int (&off)[K]) {
    P.tx_interior = 0;
    P.tx_halo = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int es = v[k].es;
      const int hb = (v[k].flags & RV_HALO) ? 16 : 0;  // halo chunk bytes
      const int xb = xs * es;
      const int c0 = max(xb - hb, 0);
      const int c1 = min(xb + 32 * V * es + hb, v[k].ld * es);
      P.nb[k] = v[k].base ? (c1 - c0) : 0;
      P.src[k] = v[k].base + c0;
      P.row_bytes[k] = (size_t)v[k].ld * (size_t)es;
      P.dst[k] = (uint32_t)(off[k] + c0 - (xb - hb));
      P.always[k] = (v[k].flags & RV_ALWAYS) != 0;
      P.tx_interior += (uint32_t)P.nb[k];
      if (P.always[k]) P.tx_halo += (uint32_t)P.nb[k];
    }
  }

  // Lane 0: issue the copies of one row into the next slot (rows are produced
  // in sequence order).  Out-of-grid rows only complete the slot's phase.
  template <int V, int K>
  __device__ __forceinline__ void produce(int row, int ny, bool interior, const Plan<V, K>& P) {
    if ((threadIdx.x & 31) != 0 || failed) return;  // after a failure nothing more is issued
    const int s = pslot;
    pslot = (pslot + 1 == S) ? 0 : pslot + 1;
    ++q_issued;
    const uint32_t bar = bars + 8u * s;
    const uint32_t dst0 = slots + (uint32_t)(s * slot_bytes);
    // the slot's previous contents were read through the generic proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (row < 0 || row >= ny) {
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
      return;
    }
    const uint32_t tx = interior ? P.tx_interior : P.tx_halo;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(tx) : "memory");
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (P.nb[k] == 0 || (!interior && !P.always[k])) continue;
      const unsigned char* src = P.src[k] + (size_t)row * P.row_bytes[k];
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              dst0 + P.dst[k]),
          "l"(src), "r"(P.nb[k]), "r"(bar)
          : "memory");
    }
  }

  // Whole warp: wait until the next row (in sequence order) has landed.
  __device__ __forceinline__ const unsigned char* wait(unsigned) {
    const int s = cslot;
    const uint32_t bar = bars + 8u * s;
    const uint32_t parity = cpar;
    if (cslot + 1 == S) {
      cslot = 0;
      cpar ^= 1u;
    } else {
      ++cslot;
    }
    if (!failed) {
      // fast path: the row has usually landed already (it was issued S rows
      // ago); the timer is read only when the first probe fails
      uint32_t ready;
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(ready)
          : "r"(bar), "r"(parity)
          : "memory");
      if (__all_sync(0xffffffffu, ready != 0u)) return slots_ptr + (size_t)s * slot_bytes;
      const unsigned long long t0 = global_ns();
      unsigned spins = 0;
      for (;;) {
        uint32_t ok;
        // a short suspend hint: a row in flight usually lands within a
        // microsecond, and a long default suspension would outlast it
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity), "r"(kSuspendHintNs)
            : "memory");
        if (ok) break;
        if ((++spins & 15u) == 0u && (long long)(global_ns() - t0) > timeout_ns) {
          failed = true;  // record once; later rows are not waited for
          if ((threadIdx.x & 31) == 0) {
            if (err) atomicCAS(err, 0, LAP5CG_ERR_SYNC_TIMEOUT);
            __threadfence();
            if (abort_flag) atomicExch(abort_flag, 1);
          }
          break;
        }
      }
      failed = __any_sync(0xffffffffu, failed);
    }
    return slots_ptr + (size_t)s * slot_bytes;
  }

  // Invalidate the barriers (every produced row has been waited for) so the
  // same shared memory can hold a fresh ring for the next solve.  After a
  // timed-out wait no new copies were issued, but earlier ones may still be in
  // flight: drain them first (bounded, 1 s per slot).
  __device__ __forceinline__ void teardown() {
    __syncwarp();
    if (failed && (threadIdx.x & 31) == 0) {
      const unsigned first = q_issued > (unsigned)S ? q_issued - (unsigned)S : 0u;
      for (unsigned seq = first; seq < q_issued; ++seq) {
        const uint32_t bar = bars + 8u * (seq % (unsigned)S);
        const uint32_t parity = (seq / (unsigned)S) & 1u;
        const unsigned long long t0 = global_ns();
        for (;;) {
          uint32_t ok;
          asm volatile(
              "{\n\t.reg .pred p;\n\t"
              "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
              "selp.u32 %0, 1, 0, p;\n\t}"
              : "=r"(ok)
              : "r"(bar), "r"(parity)
              : "memory");
          if (ok || global_ns() - t0 > 1000000000ull) break;
        }
      }
    }
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
      for (int s = 0; s < S; ++s) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bars + 8u * s) : "memory");
    }
    __syncwarp();
  }

  __device__ __forceinline__ void fence_global_to_async() {
    if ((threadIdx.x & 31) == 0) asm volatile("fence.proxy.async.global;" ::: "memory");
  }
};

// Lane view of one ring slot.  Vector k's segment starts at off[k]; with a
// halo the lane's first element sits 16 bytes further.
template <int V, class T, class M>
__device__ __forceinline__ void ring_lane(const unsigned char* slot, int off, bool halo, int lane, int x, int nx,
                                          M (&v)[V]) {
  using U = typename std::remove_const<T>::type;
  using L = Lanes<V>;
  const U* p = reinterpret_cast<const U*>(slot + off + (halo ? 16 : 0)) + lane * L::W;
  if constexpr (L::G == 1) {
    load_group<V, U, M>(p, x, nx, v);
  } else {
#pragma unroll
    for (int gi = 0; gi < L::G; ++gi) {
      M t[L::W];
      load_group<L::W, U, M>(p + gi * L::GS, x + gi * L::GS, nx, t);
#pragma unroll
      for (int k = 0; k < L::W; ++k) v[gi * L::W + k] = t[k];
    }
  }
}

// Halo columns of a stencil operand: left (column xs-1) for lane 0, right
// (column xs+32V) for lane 31, 0 outside [0, nx).
template <int V, class T, class M>
__device__ __forceinline__ M ring_halo(const unsigned char* slot, int off, int lane, int xs, int nx) {
  using U = typename std::remove_const<T>::type;
  const U* p = reinterpret_cast<const U*>(slot + off);
  constexpr int h = 16 / (int)sizeof(U);
  if (lane == 0) return (xs - 1 >= 0 && xs - 1 < nx) ? to_math<M, U>(p[h - 1]) : M(0);
  if (lane == 31) return (xs + 32 * V < nx) ? to_math<M, U>(p[h + 32 * V]) : M(0);
  return M(0);
}

// Row march of one unit through the ring: rows y0-1 .. y1 (or reversed) are
// streamed; field(j, slot, FRow&) builds the stencil operand of row j from its
// slot, finish(j, slot, S, C, N) consumes row j.  Whole-warp call.
template <int V, class M, int K, class FieldF, class FinishF>
__device__ __forceinline__ void march_ring(WarpRing& ring, int ny, int xs, int y0, int y1, bool rev,
                                           const RingVec (&vecs)[K], const int (&off)[K], FieldF& field,
                                           FinishF& finish) {
  if (y0 >= y1) return;
  const int T = y1 - y0;
  const int step = rev ? -1 : 1;
  const int ystart = rev ? y1 - 1 : y0;
  const unsigned q0 = ring.q;
  auto row_of = [&](int t) { return ystart + (t - 1) * step; };
  const int total = T + 2;
  const int pre = min(ring.S, total);
  typename WarpRing::Plan<V, K> P;
  WarpRing::plan<V, K>(P, xs, vecs, off);
  for (int t = 0; t < pre; ++t) ring.produce<V, K>(row_of(t), ny, t >= 1 && t <= T, P);
  FRow<V, M> fB, fC;
  {
    const unsigned char* s0 = ring.wait(q0);
    if (row_of(0) < 0 || row_of(0) >= ny) fB.zero(); else field(row_of(0), s0, fB);
    __syncwarp();
    if (ring.S < total) ring.produce<V, K>(row_of(ring.S), ny, ring.S <= T, P);
  }
  const unsigned char* sC = ring.wait(q0 + 1);
  field(row_of(1), sC, fC);
  for (int t = 1; t <= T; ++t) {
    FRow<V, M> fA;
    const unsigned char* sA = ring.wait(q0 + t + 1);
    if (row_of(t + 1) < 0 || row_of(t + 1) >= ny) fA.zero(); else field(row_of(t + 1), sA, fA);
    if (!rev) finish(row_of(t), sC, fB, fC, fA);
    else finish(row_of(t), sC, fA, fC, fB);
    __syncwarp();
    if (t + ring.S < total) ring.produce<V, K>(row_of(t + ring.S), ny, t + ring.S <= T, P);
    fB = fC;
    fC = fA;
    sC = sA;
  }
  ring.q = q0 + (unsigned)total;
}

// Element-wise variant (no stencil operand): rows y0 .. y1-1 only.
template <int V, int K, class FinishF>
__device__ __forceinline__ void stream_ring(WarpRing& ring, int ny, int xs, int y0, int y1, bool rev,
                                            const RingVec (&vecs)[K], const int (&off)[K], FinishF& finish) {
  if (y0 >= y1) return;
  const int T = y1 - y0;
  const int step = rev ? -1 : 1;
  const int ystart = rev ? y1 - 1 : y0;
  const unsigned q0 = ring.q;
  const int pre = min(ring.S, T);
  typename WarpRing::Plan<V, K> P;
  WarpRing::plan<V, K>(P, xs, vecs, off);
  for (int t = 0; t < pre; ++t) ring.produce<V, K>(ystart + t * step, ny, true, P);
  for (int t = 0; t < T; ++t) {
    const unsigned char* sl = ring.wait(q0 + t);
    finish(ystart + t * step, sl);
    __syncwarp();
    if (t + ring.S < T) ring.produce<V, K>(ystart + (t + ring.S) * step, ny, true, P);
  }
  ring.q = q0 + (unsigned)T;
}

// Byte offsets of K vectors inside a slot, each segment a multiple of 16 bytes.
template <int V, int K>
__host__ __device__ inline int ring_layout(const RingVec (&v)[K], int (&off)[K]) {
  int o = 0;
  for (int k = 0; k < K; ++k) {
    off[k] = o;
    o += ring_seg_bytes(V, v[k].es, (v[k].flags & RV_HALO) != 0);
  }
  return o;
}

}  // namespace lap5
