// small.cu -- cluster-resident solves for small grids (the paper's own sizes,
// N = 16 .. ~250): the whole grid lives in the shared memory of one
// thread-block cluster of up to 16 CTAs.
//
// CTA c of the cluster owns a contiguous block of rows of every state vector
// in its shared memory, with one halo row above and below.  After a stencil
// operand is updated, each CTA writes its first and last rows into the halo
// rows of its neighbours through distributed shared memory; a cluster barrier
// publishes them.  Dot products are reduced through distributed shared memory
// in a fixed order (every CTA gets bit-identical scalars).  Global memory is
// touched only to load b and x0 and to store x.  Arithmetic and order are
// those of the streaming kernels: Algorithm 1 (z = A p stored, as in
// binary64) and Algorithm 2, fixed stencil add order, FMA axpys, FP64 dot
// products (binary32: Dot2).
#include <algorithm>
#include <cooperative_groups.h>
#include <vector>

#include "cg_kernels.cuh"
#include "launch.h"

namespace lap5 {

namespace cgx = cooperative_groups;

template <class T>
struct SmallArgs {
  int nx, ny, ld;   // grid and global pitch
  int R;            // most rows any CTA owns
  int ldp;          // shared-memory row pitch (elements)
  const T* b;
  T* x;
  lap5cg_info* info;
  double* history;
  double tol;
  int maxit;
  int true_res;
  int variant;
};

// Rows of CTA c when ny rows are split over C CTAs as evenly as possible.
__device__ __forceinline__ void small_rows(int ny, int C, int c, int& r0, int& nr) {
  const int q = ny / C, rem = ny % C;
  nr = q + (c < rem ? 1 : 0);
  r0 = c * q + (c < rem ? c : rem);
}

// Cluster reduction of NV values (per-thread contributions): warp shuffle
// tree, CTA partial, then every CTA reads all CTA partials through distributed
// shared memory in rank order.  Parity-double-buffered slots.
// No scalar follow-up (see the overload below).
struct NoPost {
  __device__ void operator()(const double*, double*) const {}
};

// Cluster reduction of NV values, then post(sums, extra) on one thread (warp
// 0, lane 0) with its NE results broadcast to the CTA with the sums: the
// scalar arithmetic of the iteration (divisions) runs once a CTA instead of
// once a thread -- on this GPU's FP64 pipe a division in every thread of a
// CTA costs microseconds.
template <int NV, int NE = 0, class Post = NoPost>
__device__ __forceinline__ void small_reduce(const double (&v)[NV], double (&out)[NV], double* red,
                                             unsigned& epoch, Post post = Post(), double* extra = nullptr) {
  static_assert(NV + NE <= kMaxVals, "reduction slots");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  auto cl = cgx::this_cluster();
  double* slot = red + 33 * kMaxVals + (int)(epoch & 1u) * kMaxVals;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp * kMaxVals + k] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = lane < nwarps ? red[lane * kMaxVals + k] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) slot[k] = s;
    }
  }
  cl.sync();
  if (warp == 0) {
    const int n = (int)cl.num_blocks();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = lane < n ? *cl.map_shared_rank(slot + k, (unsigned)lane) : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) red[32 * kMaxVals + k] = s;
    }
    if constexpr (NE > 0)
      if (lane == 0) post(red + 32 * kMaxVals, red + 32 * kMaxVals + NV);
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = red[32 * kMaxVals + k];
  if constexpr (NE > 0)
#pragma unroll
    for (int k = 0; k < NE; ++k) extra[k] = red[32 * kMaxVals + NV + k];
  __syncthreads();
  ++epoch;
}

// The cluster barrier split in two (PTX barrier.cluster): arrive with release
// semantics (this thread's earlier shared / distributed-shared writes become
// visible to every thread that has waited), wait with acquire semantics.
// Work placed between the two overlaps the barrier's latency.
// Every thread of the cluster calls both, once per phase; the .aligned forms
// need the warp converged, hence the __syncwarp.
__device__ __forceinline__ void cluster_arrive_release() {
  __syncwarp();
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
  __syncwarp();
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// Pipelined NewCG exchange area of a CTA (after the vectors in dynamic shared
// memory): the w halo rows and the CTA partials of (gamma, delta), both
// double-buffered by iteration parity.  Neighbours write the halo rows and
// every CTA writes its partials into every CTA's slots, so that after the
// barrier each CTA reads them from its own shared memory.
template <class T>
struct SmallXchg {
  T* halo;        // [2 parities][2: above, below][ldp]
  double* slots;  // [2 parities][kMaxCtas16][2]
  int ldp;
  __device__ __forceinline__ T* row(int par, int below) const { return halo + (size_t)(2 * par + below) * ldp; }
  __device__ __forceinline__ double* slot(int par, int rank) const { return slots + (size_t)(par * 16 + rank) * 2; }
};

// CTA sum of two per-thread values (warp shuffle tree, then warp 0 over the
// warps), stored into slot(par, my rank) of every CTA of the cluster.
__device__ __forceinline__ void small_publish2(double v0, double v1, const SmallXchg<double>& xs_d, int par,
                                               int rank, int C, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v0 += __shfl_xor_sync(0xffffffffu, v0, o);
    v1 += __shfl_xor_sync(0xffffffffu, v1, o);
  }
  if (lane == 0) {
    red[warp * kMaxVals + 0] = v0;
    red[warp * kMaxVals + 1] = v1;
  }
  __syncthreads();
  if (warp == 0) {
    double s0 = lane < nwarps ? red[lane * kMaxVals + 0] : 0.0;
    double s1 = lane < nwarps ? red[lane * kMaxVals + 1] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    if (lane < C) {
      auto cl = cgx::this_cluster();
      double* dst = cl.map_shared_rank(xs_d.slot(par, rank), (unsigned)lane);
      dst[0] = s0;
      dst[1] = s1;
    }
  }
}

template <class T>
struct SmallView {
  T* base;   // this CTA's shared memory for vector 0
  int rows;  // R + 2 (halo rows at local -1 and R)
  int ldp;
  __device__ __forceinline__ T* vec(int v) const { return base + (size_t)v * rows * ldp; }
  // element (local row i in [-1, R], column k) of vector v
  __device__ __forceinline__ T& at(int v, int i, int k) const { return vec(v)[(size_t)(i + 1) * ldp + k]; }
};

// y = A g on the CTA's own rows (g has its halo rows filled); fixed add order.
template <class T, class M>
__device__ __forceinline__ M small_stencil(const SmallView<T>& sv, int g, int i, int k, int nx) {
  const M c = to_math<M, T>(sv.at(g, i, k));
  const M w = k > 0 ? to_math<M, T>(sv.at(g, i, k - 1)) : M(0);
  const M e = k + 1 < nx ? to_math<M, T>(sv.at(g, i, k + 1)) : M(0);
  const M s = to_math<M, T>(sv.at(g, i - 1, k));
  const M n = to_math<M, T>(sv.at(g, i + 1, k));
  M acc = M(4) * c;
  acc -= w;
  acc -= e;
  acc -= s;
  acc -= n;
  return acc;
}

// Write this CTA's first / last own rows of vector g into the neighbours' halo
// rows (distributed shared memory); the caller's cluster barrier publishes them.
template <class T>
__device__ __forceinline__ void small_push(const SmallView<T>& sv, int g, int nr, int nx, int rank, int C, int ny) {
  auto cl = cgx::this_cluster();
  const int tid = threadIdx.x, nt = blockDim.x;
  if (rank > 0) {
    int r0p, nrp;
    small_rows(ny, C, rank - 1, r0p, nrp);
    T* dst = cl.map_shared_rank(&sv.at(g, nrp, 0), (unsigned)(rank - 1));  // its bottom halo row
    for (int k = tid; k < nx; k += nt) dst[k] = sv.at(g, 0, k);
  }
  if (rank + 1 < C) {
    T* dst = cl.map_shared_rank(&sv.at(g, -1, 0), (unsigned)(rank + 1));  // its top halo row
    for (int k = tid; k < nx; k += nt) dst[k] = sv.at(g, nr - 1, k);
  }
}

// vector slots in shared memory
enum { SV_B = 0, SV_X, SV_R, SV_P, SV_Z, SV_W, SV_Q, SV_N, SV_COUNT_CLASSIC = 5, SV_COUNT_NEWCG = 8 };

// Bytes of the NewCG exchange area (w halo rows and partial slots).
__host__ __device__ inline size_t small_xchg_bytes(int ldp, size_t es) {
  return align_up((size_t)4 * ldp * es, 16) + (size_t)2 * 16 * 2 * sizeof(double);
}

// One cluster-resident solve (the whole body of the kernels below).  red and
// scal are static shared memory of the calling kernel (scal: NewCG's gamma,
// delta, alpha, beta and continue / stop / status), dsm its dynamic shared
// memory.
template <class T>
__device__ __forceinline__ void small_body(const SmallArgs<T>& a, double* red, double* scal, unsigned char* dsm) {
  using M = typename Math<T>::type;
  using Acc = typename AccOf<M>::type;
  auto cl = cgx::this_cluster();
  const int rank = (int)cl.block_rank(), C = (int)cl.num_blocks();
  int r0, nr;
  small_rows(a.ny, C, rank, r0, nr);
  const int nx = a.nx, ny = a.ny;
  const SmallView<T> sv{reinterpret_cast<T*>(dsm), a.R + 2, a.ldp};
  const int nvec = a.variant == LAP5CG_NEWCG ? SV_COUNT_NEWCG : SV_COUNT_CLASSIC;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int npts = nr * nx;
  unsigned epoch = 0;

  // zero everything (halo rows at the grid edge stay zero), load b and x0
  for (int v = 0; v < nvec; ++v)
    for (int e = tid; e < sv.rows * sv.ldp; e += nt) sv.vec(v)[e] = from_math<T, M>(M(0));
  SmallXchg<T> xh;
  SmallXchg<double> xd;
  {
    unsigned char* xbase = dsm + (size_t)nvec * sv.rows * sv.ldp * sizeof(T);
    xh.halo = reinterpret_cast<T*>(xbase);
    xh.ldp = sv.ldp;
    xd.slots = reinterpret_cast<double*>(xbase + align_up((size_t)4 * sv.ldp * sizeof(T), 16));
    xd.ldp = sv.ldp;
    xh.slots = xd.slots;
    if (a.variant == LAP5CG_NEWCG) {
      for (int e = tid; e < 4 * sv.ldp; e += nt) xh.halo[e] = from_math<T, M>(M(0));
      for (int e = tid; e < 2 * 16 * 2; e += nt) xd.slots[e] = 0.0;
    }
  }
  __syncthreads();
  for (int e = tid; e < npts; e += nt) {
    const int i = e / nx, k = e - i * nx;
    sv.at(SV_B, i, k) = a.b[(size_t)(r0 + i) * a.ld + k];
    sv.at(SV_X, i, k) = a.x[(size_t)(r0 + i) * a.ld + k];
  }
  __syncthreads();
  small_push<T>(sv, SV_X, nr, nx, rank, C, ny);
  cl.sync();

  int status = LAP5CG_NOT_CONVERGED, iters = 0;
  double bb, gamma, delta = 0.0, relres_true = nan("");
  {  // r = b - A x0, (b, b), (r, r)
    Acc abb, arr;
    for (int e = tid; e < npts; e += nt) {
      const int i = e / nx, k = e - i * nx;
      const M bv = to_math<M, T>(sv.at(SV_B, i, k));
      const M rv = bv - small_stencil<T, M>(sv, SV_X, i, k, nx);
      sv.at(SV_R, i, k) = from_math<T, M>(rv);
      abb.add(bv, bv);
      arr.add(rv, rv);
    }
    double v[2] = {abb.value(), arr.value()}, o[2];
    small_reduce<2>(v, o, red, epoch);
    bb = o[0];
    gamma = o[1];
  }
  bool store_x = false;
  if (!isfinite(bb)) {
    status = LAP5CG_ERR_NONFINITE;
    gamma = 0.0;
    goto done;
  }
  if (bb == 0.0) {
    for (int e = tid; e < npts; e += nt) sv.at(SV_X, e / nx, e % nx) = from_math<T, M>(M(0));
    status = LAP5CG_OK;
    relres_true = 0.0;
    store_x = true;
    goto done;
  }
  store_x = true;
  {
    const double thr = a.tol > 0.0 ? a.tol * a.tol * bb : 0.0;
    if (a.variant != LAP5CG_NEWCG) {
      // ------------------------------ Algorithm 1 ------------------------------
      if (a.history && rank == 0 && tid == 0) a.history[0] = sqrt(gamma / bb);
      if (!isfinite(gamma)) { status = LAP5CG_ERR_NONFINITE; goto truecheck; }
      if (gamma <= thr) { status = LAP5CG_OK; goto truecheck; }
      double beta = 0.0, alpha_bc = 0.0, beta_bc = 0.0;
      while (iters < a.maxit) {
        const M bm = (M)beta;
        for (int e = tid; e < npts; e += nt) {  // p = r + beta p
          const int i = e / nx, k = e - i * nx;
          const M rv = to_math<M, T>(sv.at(SV_R, i, k));
          sv.at(SV_P, i, k) = from_math<T, M>(iters == 0 ? rv : fmx(bm, to_math<M, T>(sv.at(SV_P, i, k)), rv));
        }
        __syncthreads();
        small_push<T>(sv, SV_P, nr, nx, rank, C, ny);
        cl.sync();
        double pz;
        {
          Acc acc;
          for (int e = tid; e < npts; e += nt) {  // z = A p, (p, z)
            const int i = e / nx, k = e - i * nx;
            const M zv = small_stencil<T, M>(sv, SV_P, i, k, nx);
            sv.at(SV_Z, i, k) = from_math<T, M>(zv);
            acc.add(to_math<M, T>(sv.at(SV_P, i, k)), zv);
          }
          double v[1] = {acc.value()}, o[1], e[1];
          const double gm = gamma;
          small_reduce<1, 1>(v, o, red, epoch, [gm](const double* sum, double* ex) { ex[0] = gm / sum[0]; }, e);
          pz = o[0];
          alpha_bc = e[0];
        }
        if (!(pz > 0.0) || !isfinite(pz)) { status = LAP5CG_ERR_BREAKDOWN; goto truecheck; }
        const double alpha = alpha_bc;
        const M am = (M)alpha;
        double gnew;
        {
          Acc acc;
          for (int e = tid; e < npts; e += nt) {  // x += alpha p, r -= alpha z, (r, r)
            const int i = e / nx, k = e - i * nx;
            sv.at(SV_X, i, k) = from_math<T, M>(fmx(am, to_math<M, T>(sv.at(SV_P, i, k)), to_math<M, T>(sv.at(SV_X, i, k))));
            const M rv = fmx(-am, to_math<M, T>(sv.at(SV_Z, i, k)), to_math<M, T>(sv.at(SV_R, i, k)));
            sv.at(SV_R, i, k) = from_math<T, M>(rv);
            acc.add(rv, rv);
          }
          double v[1] = {acc.value()}, o[1], e[1];
          const double gm = gamma;
          small_reduce<1, 1>(v, o, red, epoch, [gm](const double* sum, double* ex) { ex[0] = sum[0] / gm; }, e);
          gnew = o[0];
          beta_bc = e[0];
        }
        ++iters;
        if (a.history && rank == 0 && tid == 0) a.history[iters] = sqrt(gnew / bb);
        if (!isfinite(gnew)) { status = LAP5CG_ERR_NONFINITE; gamma = gnew; goto truecheck; }
        beta = beta_bc;
        gamma = gnew;
        if (gnew <= thr) { status = LAP5CG_OK; goto truecheck; }
      }
    } else {
      // ------------------------------ Algorithm 2 ------------------------------
      // One cluster barrier per iteration, split into arrive and wait: a CTA
      // publishes its (gamma, delta) partials and its new w boundary rows,
      // arrives, computes n = A w on the rows that need no neighbour row, and
      // only then waits -- the reduction overlaps the stencil (Sec. II, Fig.
      // NewCG).  The remaining rows of n, the scalars and the six pointwise
      // updates follow the wait.  Halo rows and partial slots alternate
      // between two buffers by iteration parity, so a CTA that runs ahead
      // never overwrites what a neighbour has yet to read.
      {  // w = A r, gamma = (r, r), delta = (w, r); publish for the first wait
        __syncthreads();
        small_push<T>(sv, SV_R, nr, nx, rank, C, ny);
        cl.sync();
        Acc ag, ad;
        for (int e = tid; e < npts; e += nt) {
          const int i = e / nx, k = e - i * nx;
          const M wv = small_stencil<T, M>(sv, SV_R, i, k, nx);
          const M rv = to_math<M, T>(sv.at(SV_R, i, k));
          sv.at(SV_W, i, k) = from_math<T, M>(wv);
          ag.add(rv, rv);
          ad.add(wv, rv);
        }
        small_publish2(ag.value(), ad.value(), xd, 0, rank, C, red);  // its __syncthreads orders the w writes
        if (rank > 0)
          for (int k = tid; k < nx; k += nt) cl.map_shared_rank(xh.row(0, 1), (unsigned)(rank - 1))[k] = sv.at(SV_W, 0, k);
        if (rank + 1 < C)
          for (int k = tid; k < nx; k += nt) cl.map_shared_rank(xh.row(0, 0), (unsigned)(rank + 1))[k] = sv.at(SV_W, nr - 1, k);
        cluster_arrive_release();
      }
      double alpha = 0.0, gold = 0.0;
      int par = 0;
      for (;;) {
        const bool first = (iters == 0);
        // n = A w on the rows whose neighbours are this CTA's own (overlaps the barrier)
        const int ni = nr > 2 ? (nr - 2) * nx : 0;
        for (int e = tid; e < ni; e += nt) {
          const int i = 1 + e / nx, k = e - (i - 1) * nx;
          sv.at(SV_N, i, k) = from_math<T, M>(small_stencil<T, M>(sv, SV_W, i, k, nx));
        }
        cluster_wait_acquire();
        if (tid < 32) {  // one warp forms the scalars while the others start the boundary rows
          const int lane = tid;
          double g = lane < C ? xd.slot(par, lane)[0] : 0.0;
          double d = lane < C ? xd.slot(par, lane)[1] : 0.0;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {  // the same tree in every CTA: identical scalars
            g += __shfl_xor_sync(0xffffffffu, g, o);
            d += __shfl_xor_sync(0xffffffffu, d, o);
          }
          if (lane == 0) {
            double st = 0.0, al = alpha, be = 0.0;  // st: 0 go on, 1 stop, or a (negative) status
            if (!isfinite(g)) {
              st = LAP5CG_ERR_NONFINITE;
            } else if (g <= thr) {
              st = 1.0;
            } else if (iters >= a.maxit) {
              st = 2.0;
            } else if (first) {
              if (!(d > 0.0) || !isfinite(d)) st = LAP5CG_ERR_BREAKDOWN;
              else al = g / d;
            } else {
              be = g / gold;
              const double denom = d / g - be / alpha;
              if (!(denom > 0.0) || !isfinite(denom)) st = LAP5CG_ERR_BREAKDOWN;
              else al = 1.0 / denom;
            }
            scal[0] = g;
            scal[1] = d;
            scal[2] = al;
            scal[3] = be;
            scal[4] = st;
            if (a.history && rank == 0) a.history[iters] = sqrt(g / bb);
          }
        }
        // n on the first and last own rows: their outer neighbours are the halo rows of this parity
        {
          const int nb = nr > 1 ? 2 * nx : nx;
          for (int e = tid; e < nb; e += nt) {
            const int i = (e < nx) ? 0 : nr - 1, k = e < nx ? e : e - nx;
            const M c = to_math<M, T>(sv.at(SV_W, i, k));
            const M w = k > 0 ? to_math<M, T>(sv.at(SV_W, i, k - 1)) : M(0);
            const M ee = k + 1 < nx ? to_math<M, T>(sv.at(SV_W, i, k + 1)) : M(0);
            const M so = to_math<M, T>(i == 0 ? xh.row(par, 0)[k] : sv.at(SV_W, i - 1, k));
            const M no = to_math<M, T>(i == nr - 1 ? xh.row(par, 1)[k] : sv.at(SV_W, i + 1, k));
            M acc = M(4) * c;
            acc -= w;
            acc -= ee;
            acc -= so;
            acc -= no;
            sv.at(SV_N, i, k) = from_math<T, M>(acc);
          }
        }
        __syncthreads();  // n and the scalars complete, every read of w done before w changes
        gamma = scal[0];
        delta = scal[1];
        const double beta = scal[3];
        {
          const double st = scal[4];
          if (st != 0.0) {
            if (st == 1.0) status = LAP5CG_OK;
            else if (st < 0.0) status = (int)st;
            goto truecheck;
          }
        }
        alpha = scal[2];
        const M am = (M)alpha, bm = (M)beta;
        Acc ag, ad;
        for (int e = tid; e < npts; e += nt) {
          const int i = e / nx, k = e - i * nx;
          const M nv = to_math<M, T>(sv.at(SV_N, i, k));
          const M wv0 = to_math<M, T>(sv.at(SV_W, i, k));
          const M rv0 = to_math<M, T>(sv.at(SV_R, i, k));
          M zv, qv, pv;
          if (first) {
            zv = nv;
            qv = wv0;
            pv = rv0;
          } else {
            zv = fmx(bm, to_math<M, T>(sv.at(SV_Z, i, k)), nv);
            qv = fmx(bm, to_math<M, T>(sv.at(SV_Q, i, k)), wv0);
            pv = fmx(bm, to_math<M, T>(sv.at(SV_P, i, k)), rv0);
          }
          // stored then re-read (rounded to T), as the streaming kernels use them
          const M zs = to_math<M, T>(from_math<T, M>(zv)), qs = to_math<M, T>(from_math<T, M>(qv));
          const M ps = to_math<M, T>(from_math<T, M>(pv));
          sv.at(SV_Z, i, k) = from_math<T, M>(zv);
          sv.at(SV_Q, i, k) = from_math<T, M>(qv);
          sv.at(SV_P, i, k) = from_math<T, M>(pv);
          sv.at(SV_X, i, k) = from_math<T, M>(fmx(am, ps, to_math<M, T>(sv.at(SV_X, i, k))));
          const M rv = fmx(-am, qs, rv0);
          const M wv = fmx(-am, zs, wv0);
          sv.at(SV_R, i, k) = from_math<T, M>(rv);
          sv.at(SV_W, i, k) = from_math<T, M>(wv);
          ag.add(rv, rv);
          ad.add(wv, rv);
        }
        ++iters;
        gold = gamma;
        par ^= 1;
        small_publish2(ag.value(), ad.value(), xd, par, rank, C, red);  // its __syncthreads orders the w writes
        if (rank > 0)
          for (int k = tid; k < nx; k += nt) cl.map_shared_rank(xh.row(par, 1), (unsigned)(rank - 1))[k] = sv.at(SV_W, 0, k);
        if (rank + 1 < C)
          for (int k = tid; k < nx; k += nt) cl.map_shared_rank(xh.row(par, 0), (unsigned)(rank + 1))[k] = sv.at(SV_W, nr - 1, k);
        cluster_arrive_release();
      }
    }
  }
truecheck:
  if (a.true_res) {
    __syncthreads();
    small_push<T>(sv, SV_X, nr, nx, rank, C, ny);
    cl.sync();
    Acc arr;
    for (int e = tid; e < npts; e += nt) {
      const int i = e / nx, k = e - i * nx;
      const M rv = to_math<M, T>(sv.at(SV_B, i, k)) - small_stencil<T, M>(sv, SV_X, i, k, nx);
      arr.add(rv, rv);
    }
    double v[1] = {arr.value()}, o[1];
    small_reduce<1>(v, o, red, epoch);
    relres_true = sqrt(o[0] / bb);
  }
done:
  __syncthreads();
  if (store_x)
    for (int e = tid; e < npts; e += nt) {
      const int i = e / nx, k = e - i * nx;
      a.x[(size_t)(r0 + i) * a.ld + k] = sv.at(SV_X, i, k);
    }
  if (rank == 0 && tid == 0) {
    lap5cg_info inf;
    inf.status = status;
    inf.iters = iters;
    inf.outer_iters = 0;
    inf.pad = 0;
    inf.relres_recursive = (bb > 0.0) ? sqrt(gamma / bb) : 0.0;
    inf.relres_true = relres_true;
    *a.info = inf;
  }
  cl.sync();  // no CTA leaves while a neighbour may still read its shared memory
}

template <class T>
__global__ void __launch_bounds__(512, 1) k_small(const SmallArgs<T> a) {
  __shared__ double red[kRedDoubles];
  __shared__ double scal[5];
  extern __shared__ __align__(16) unsigned char dsm[];
  small_body<T>(a, red, scal, dsm);
}

// Many small instances in one launch: cluster i of the grid solves instance i
// (batched solves of grids that fit in one cluster's shared memory).
constexpr int kSmallBatchMax = 96;
template <class T>
struct SmallBatchArgs {
  int C;  // CTAs per cluster (= per instance)
  int n;  // instances in this launch
  SmallArgs<T> a[kSmallBatchMax];
};

template <class T>
__global__ void __launch_bounds__(512, 1) k_small_batch(const SmallBatchArgs<T> sb) {
  __shared__ double red[kRedDoubles];
  __shared__ double scal[5];
  extern __shared__ __align__(16) unsigned char dsm[];
  const int i = (int)blockIdx.x / sb.C;
  if (i < sb.n) small_body<T>(sb.a[i], red, scal, dsm);  // whole clusters take the same branch
}

// Shared memory a cluster-resident solve needs per CTA (0 if it does not fit).
template <class T>
static size_t small_smem(int nx, int ny, int variant, int C, int* R_out, int* ldp_out) {
  const int R = (ny + C - 1) / C;
  const int ldp = (nx + 1) / 2 * 2;
  const int nvec = variant == LAP5CG_NEWCG ? SV_COUNT_NEWCG : SV_COUNT_CLASSIC;
  *R_out = R;
  *ldp_out = ldp;
  const size_t vec_bytes = (size_t)nvec * (R + 2) * ldp * sizeof(T);
  return variant == LAP5CG_NEWCG ? vec_bytes + small_xchg_bytes(ldp, sizeof(T)) : vec_bytes;
}

template <class T>
static int try_small_t(const SolvePlan& p, cudaStream_t st, bool* used) {
  *used = false;
  // an explicit march choice or residual replacement asks for the streaming kernels
  if (p.opts.resident < 0 || p.opts.ring_slots != 0 || p.opts.rr_period > 0 || p.opts.reproducible ||
      p.opts.stabilized)
    return LAP5CG_OK;
  DevProps dp;
  int rc = dev_props(&dp);
  if (rc != LAP5CG_OK) return rc;
  // one to sixteen CTAs (team_ctas, default 16), each at least one row
  int C = p.opts.team_ctas;
  if (C != 1 && C != 2 && C != 4 && C != 8 && C != 16) C = 16;
  if (C > p.ny) C = p.ny;
  int R, ldp;
  const size_t smem = small_smem<T>(p.nx, p.ny, p.variant, C, &R, &ldp);
  if (smem + sizeof(double) * kRedDoubles + 1024 > (size_t)dp.max_smem_optin) return LAP5CG_OK;  // too large
  const void* fn = reinterpret_cast<const void*>(&k_small<T>);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return LAP5CG_ERR_CUDA;
  if (C > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return LAP5CG_ERR_CUDA;
  SmallArgs<T> a;
  a.nx = p.nx;
  a.ny = p.ny;
  a.ld = p.ld;
  a.R = R;
  a.ldp = ldp;
  a.b = static_cast<const T*>(p.b);
  a.x = static_cast<T*>(p.x);
  a.info = p.info;
  a.history = p.opts.history;
  a.tol = p.tol;
  a.maxit = p.maxit;
  a.true_res = p.opts.true_residual;
  a.variant = p.variant;
  cudaLaunchConfig_t lc = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  lc.gridDim = dim3(C);
  lc.blockDim = dim3(32 * (p.opts.warps_per_cta > 0 ? p.opts.warps_per_cta : 8));
  lc.dynamicSmemBytes = smem;
  lc.stream = st;
  lc.attrs = attr;
  lc.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &lc) != cudaSuccess || nclusters < 1) {
    cudaGetLastError();
    return LAP5CG_OK;  // this cluster shape cannot run here: use the streaming kernels
  }
  void* args[] = {&a};
  if (cudaLaunchKernelExC(&lc, fn, args) != cudaSuccess) return LAP5CG_ERR_CUDA;
  *used = true;
  return LAP5CG_OK;
}

// Batched solves: instances of F64 / F32 shape that fit in one cluster's
// shared memory (and at least one row a CTA) are solved by k_small_batch, one
// cluster an instance, kSmallBatchMax a launch; taken[k] marks them.  The
// options that ask for the streaming kernels for single solves do so here.
template <class T>
static int small_batched_t(int count, const int* nx, const int* ny, const int* ld, const void* const* b,
                           void* const* x, double tol, int maxit, int variant, lap5cg_info* info,
                           const lap5cg_opts& o, cudaStream_t st, std::vector<char>& taken) {
  if (o.resident < 0 || o.ring_slots != 0 || o.rr_period > 0 || o.reproducible || o.stabilized) return LAP5CG_OK;
  DevProps dp;
  int rc = dev_props(&dp);
  if (rc != LAP5CG_OK) return rc;
  int C = o.team_ctas;
  if (C != 1 && C != 2 && C != 4 && C != 8 && C != 16) C = 16;
  const int wpc = o.warps_per_cta > 0 ? (o.warps_per_cta > 16 ? 16 : o.warps_per_cta) : 8;
  std::vector<int> pick;
  std::vector<SmallArgs<T>> args;
  size_t smem_max = 0;
  for (int k = 0; k < count; ++k) {
    if (ny[k] < C) continue;
    int R, ldp;
    const size_t smem = small_smem<T>(nx[k], ny[k], variant, C, &R, &ldp);
    if (smem + sizeof(double) * kRedDoubles + 1024 > (size_t)dp.max_smem_optin) continue;
    SmallArgs<T> a;
    a.nx = nx[k];
    a.ny = ny[k];
    a.ld = ld[k];
    a.R = R;
    a.ldp = ldp;
    a.b = static_cast<const T*>(b[k]);
    a.x = static_cast<T*>(x[k]);
    a.info = info + k;
    a.history = nullptr;
    a.tol = tol;
    a.maxit = maxit;
    a.true_res = o.true_residual;
    a.variant = variant;
    args.push_back(a);
    pick.push_back(k);
    if (smem > smem_max) smem_max = smem;
  }
  if (pick.empty()) return LAP5CG_OK;
  const void* fn = reinterpret_cast<const void*>(&k_small_batch<T>);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max) != cudaSuccess)
    return LAP5CG_ERR_CUDA;
  if (C > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return LAP5CG_ERR_CUDA;
  cudaLaunchConfig_t lc = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  lc.gridDim = dim3(C);
  lc.blockDim = dim3(32 * wpc);
  lc.dynamicSmemBytes = smem_max;
  lc.stream = st;
  lc.attrs = attr;
  lc.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &lc) != cudaSuccess || nclusters < 1) {
    cudaGetLastError();
    return LAP5CG_OK;  // this cluster shape cannot run here: the persistent kernel takes them all
  }
  for (size_t first = 0; first < pick.size(); first += kSmallBatchMax) {
    SmallBatchArgs<T> sb;
    sb.C = C;
    sb.n = (int)std::min<size_t>(kSmallBatchMax, pick.size() - first);
    for (int i = 0; i < sb.n; ++i) sb.a[i] = args[first + i];
    lc.gridDim = dim3(sb.n * C);
    void* kargs[] = {&sb};
    if (cudaLaunchKernelExC(&lc, fn, kargs) != cudaSuccess) return LAP5CG_ERR_CUDA;
    for (int i = 0; i < sb.n; ++i) taken[pick[first + i]] = 1;
  }
  return LAP5CG_OK;
}

int small_batched(int count, const int* nx, const int* ny, const int* ld, const void* const* b, void* const* x,
                  double tol, int maxit, int variant, int precision, lap5cg_info* info, const lap5cg_opts& o,
                  cudaStream_t st, std::vector<char>& taken) {
  taken.assign(count, 0);
  if (precision == LAP5CG_PREC_F64)
    return small_batched_t<double>(count, nx, ny, ld, b, x, tol, maxit, variant, info, o, st, taken);
  if (precision == LAP5CG_PREC_F32)
    return small_batched_t<float>(count, nx, ny, ld, b, x, tol, maxit, variant, info, o, st, taken);
  return LAP5CG_OK;
}

int try_small(const SolvePlan& p, cudaStream_t st, bool* used) {
  if (p.precision == LAP5CG_PREC_F64) return try_small_t<double>(p, st, used);
  if (p.precision == LAP5CG_PREC_F32) return try_small_t<float>(p, st, used);
  *used = false;
  return LAP5CG_OK;
}

}  // namespace lap5
