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
#include <cooperative_groups.h>

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
template <int NV>
__device__ __forceinline__ void small_reduce(const double (&v)[NV], double (&out)[NV], double* red,
                                             unsigned& epoch) {
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
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = red[32 * kMaxVals + k];
  __syncthreads();
  ++epoch;
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
enum { SV_B = 0, SV_X, SV_R, SV_P, SV_Z, SV_W, SV_Q, SV_COUNT_CLASSIC = 5, SV_COUNT_NEWCG = 7 };

template <class T>
__global__ void __launch_bounds__(512) k_small(const SmallArgs<T> a) {
  using M = typename Math<T>::type;
  using Acc = typename AccOf<M>::type;
  __shared__ double red[kRedDoubles];
  extern __shared__ __align__(16) unsigned char dsm[];
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
      double beta = 0.0;
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
          double v[1] = {acc.value()}, o[1];
          small_reduce<1>(v, o, red, epoch);
          pz = o[0];
        }
        if (!(pz > 0.0) || !isfinite(pz)) { status = LAP5CG_ERR_BREAKDOWN; goto truecheck; }
        const double alpha = gamma / pz;
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
          double v[1] = {acc.value()}, o[1];
          small_reduce<1>(v, o, red, epoch);
          gnew = o[0];
        }
        ++iters;
        if (a.history && rank == 0 && tid == 0) a.history[iters] = sqrt(gnew / bb);
        if (!isfinite(gnew)) { status = LAP5CG_ERR_NONFINITE; gamma = gnew; goto truecheck; }
        beta = gnew / gamma;
        gamma = gnew;
        if (gnew <= thr) { status = LAP5CG_OK; goto truecheck; }
      }
    } else {
      // ------------------------------ Algorithm 2 ------------------------------
      {  // w = A r, gamma = (r, r), delta = (w, r)
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
        double v[2] = {ag.value(), ad.value()}, o[2];
        small_reduce<2>(v, o, red, epoch);
        gamma = o[0];
        delta = o[1];
      }
      if (a.history && rank == 0 && tid == 0) a.history[0] = sqrt(gamma / bb);
      if (!isfinite(gamma)) { status = LAP5CG_ERR_NONFINITE; goto truecheck; }
      if (gamma <= thr) { status = LAP5CG_OK; goto truecheck; }
      if (a.maxit <= 0) goto truecheck;
      if (!(delta > 0.0) || !isfinite(delta)) { status = LAP5CG_ERR_BREAKDOWN; goto truecheck; }
      double alpha = gamma / delta, beta = 0.0;
      for (;;) {
        const bool first = (iters == 0);
        const M am = (M)alpha, bm = (M)beta;
        __syncthreads();
        small_push<T>(sv, SV_W, nr, nx, rank, C, ny);
        cl.sync();
        // stage 1: n = A w (reads w on the own rows and halos) and the
        // pointwise z, q, p recurrences
        for (int e = tid; e < npts; e += nt) {
          const int i = e / nx, k = e - i * nx;
          const M nv = small_stencil<T, M>(sv, SV_W, i, k, nx);
          const M wv = to_math<M, T>(sv.at(SV_W, i, k));
          const M rv = to_math<M, T>(sv.at(SV_R, i, k));
          M zv, qv, pv;
          if (first) {
            zv = nv;
            qv = wv;
            pv = rv;
          } else {
            zv = fmx(bm, to_math<M, T>(sv.at(SV_Z, i, k)), nv);
            qv = fmx(bm, to_math<M, T>(sv.at(SV_Q, i, k)), wv);
            pv = fmx(bm, to_math<M, T>(sv.at(SV_P, i, k)), rv);
          }
          sv.at(SV_Z, i, k) = from_math<T, M>(zv);
          sv.at(SV_Q, i, k) = from_math<T, M>(qv);
          sv.at(SV_P, i, k) = from_math<T, M>(pv);
        }
        __syncthreads();  // every stencil read of w is done before w changes
        Acc ag, ad;
        for (int e = tid; e < npts; e += nt) {
          const int i = e / nx, k = e - i * nx;
          const M pv = to_math<M, T>(sv.at(SV_P, i, k));
          const M qv = to_math<M, T>(sv.at(SV_Q, i, k));
          const M zv = to_math<M, T>(sv.at(SV_Z, i, k));
          sv.at(SV_X, i, k) = from_math<T, M>(fmx(am, pv, to_math<M, T>(sv.at(SV_X, i, k))));
          const M rv = fmx(-am, qv, to_math<M, T>(sv.at(SV_R, i, k)));
          const M wv = fmx(-am, zv, to_math<M, T>(sv.at(SV_W, i, k)));
          sv.at(SV_R, i, k) = from_math<T, M>(rv);
          sv.at(SV_W, i, k) = from_math<T, M>(wv);
          ag.add(rv, rv);
          ad.add(wv, rv);
        }
        double v[2] = {ag.value(), ad.value()}, o[2];
        small_reduce<2>(v, o, red, epoch);
        ++iters;
        if (a.history && rank == 0 && tid == 0) a.history[iters] = sqrt(o[0] / bb);
        const double gold = gamma;
        gamma = o[0];
        delta = o[1];
        if (!isfinite(gamma)) { status = LAP5CG_ERR_NONFINITE; goto truecheck; }
        if (gamma <= thr) { status = LAP5CG_OK; goto truecheck; }
        if (iters >= a.maxit) break;
        beta = gamma / gold;
        const double denom = delta / gamma - beta / alpha;
        if (!(denom > 0.0) || !isfinite(denom)) { status = LAP5CG_ERR_BREAKDOWN; goto truecheck; }
        alpha = 1.0 / denom;
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

// Shared memory a cluster-resident solve needs per CTA (0 if it does not fit).
template <class T>
static size_t small_smem(int nx, int ny, int variant, int C, int* R_out, int* ldp_out) {
  const int R = (ny + C - 1) / C;
  const int ldp = (nx + 1) / 2 * 2;
  const int nvec = variant == LAP5CG_NEWCG ? SV_COUNT_NEWCG : SV_COUNT_CLASSIC;
  *R_out = R;
  *ldp_out = ldp;
  return (size_t)nvec * (R + 2) * ldp * sizeof(T);
}

template <class T>
static int try_small_t(const SolvePlan& p, cudaStream_t st, bool* used) {
  *used = false;
  // an explicit march choice or residual replacement asks for the streaming kernels
  if (p.opts.resident < 0 || p.opts.ring_slots != 0 || p.opts.rr_period > 0 || p.opts.reproducible) return LAP5CG_OK;
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

int try_small(const SolvePlan& p, cudaStream_t st, bool* used) {
  if (p.precision == LAP5CG_PREC_F64) return try_small_t<double>(p, st, used);
  if (p.precision == LAP5CG_PREC_F32) return try_small_t<float>(p, st, used);
  *used = false;
  return LAP5CG_OK;
}

}  // namespace lap5
