// batched.cu -- cg_solve_batched: many independent grids of different shapes
// in one persistent launch.
//
// A team is one thread-block cluster (1, 2, 4, 8 or 16 CTAs).  Teams pull the
// next instance from an atomic queue over a table sorted by estimated work
// (largest first: grid points x (nx + ny), since CG iterations grow with the
// side length), solve it with the same fused passes as the single-grid
// kernels -- cluster barrier and distributed-shared-memory reductions instead
// of the grid barrier -- and move on.  An instance that converges stops by
// itself (per-instance convergence masking); its team takes the next one.
// The table is written into the workspace by small fill kernels so that the
// whole call is stream-ordered device work (capturable in a CUDA graph).
#include <algorithm>
#include <vector>

#include "ir_kernels.cuh"
#include "cg_launch.cuh"

namespace lap5 {

struct BatchEntry {
  const void* b;
  void* x;
  long long ws_off;  // byte offset of this instance's vectors in the workspace
  int nx, ny, ld;
  int idx;           // position in the caller's arrays (info slot)
};

struct BatchCtl {
  unsigned int next;  // queue head
  int pad[63];
};

struct BatchArgs {
  RingGeom rg;
  int* errs;  // per-instance error words (caller order)
  int count;
  const BatchEntry* tab;
  BatchCtl* bctl;
  unsigned char* ws;
  lap5cg_info* info;
  double tol;
  int maxit;
  int min_rows;
  int true_res;
  int store_z;
  int rr_period;
  int max_outer;
  int maxit_inner;
  double tol_inner;
};

constexpr int kFillChunk = 64;
struct FillArgs {
  BatchEntry* dst;
  int first, n;
  BatchEntry e[kFillChunk];
};

__global__ void k_fill_table(const FillArgs a) {
  const int i = threadIdx.x;
  if (i < a.n) a.dst[a.first + i] = a.e[i];
}

// Solve-kind tags.
enum { KIND_F64_CLASSIC = 0, KIND_F64_NEWCG, KIND_F32_CLASSIC, KIND_F32_NEWCG, KIND_IR_F32, KIND_IR_BF16 };

__host__ __device__ inline size_t vec_bytes(int ny, int ld, size_t es) { return align_up((size_t)ny * ld * es, kAlign); }
__host__ __device__ inline int ir_ld(int nx) { return (nx + 7) / 8 * 8; }

// Workspace bytes of one instance for a solve kind.
__host__ __device__ inline size_t instance_bytes(int kind, int nx, int ny, int ld) {
  switch (kind) {
    case KIND_F64_CLASSIC: return 4 * vec_bytes(ny, ld, 8);
    case KIND_F64_NEWCG: return 6 * vec_bytes(ny, ld, 8);
    case KIND_F32_CLASSIC: return 4 * vec_bytes(ny, ld, 4);
    case KIND_F32_NEWCG: return 6 * vec_bytes(ny, ld, 4);
    case KIND_IR_F32: return 3 * vec_bytes(ny, ir_ld(nx), 4) + 2 * vec_bytes(ny, ir_ld(nx), 4);
    default: return 3 * vec_bytes(ny, ir_ld(nx), 2) + 2 * vec_bytes(ny, ir_ld(nx), 4);
  }
}

template <int KIND> struct KindTraits;
template <> struct KindTraits<KIND_F64_CLASSIC> { using T = double; static constexpr int V = 2; };
template <> struct KindTraits<KIND_F64_NEWCG> { using T = double; static constexpr int V = 2; };
template <> struct KindTraits<KIND_F32_CLASSIC> { using T = float; static constexpr int V = 4; };
template <> struct KindTraits<KIND_F32_NEWCG> { using T = float; static constexpr int V = 4; };
template <> struct KindTraits<KIND_IR_F32> { using T = float; static constexpr int V = 4; };
template <> struct KindTraits<KIND_IR_BF16> { using T = bf16s; static constexpr int V = 4; };

// Eight columns a lane for an instance of width nx: the strips of 256 columns
// (padded width w8) cost about 0.8 of four-column strips (w4) per column.
__device__ __forceinline__ bool ir_wide(int nx) {
  const int w8 = (nx + 255) / 256 * 256, w4 = (nx + 127) / 128 * 128;
  return 4 * w8 < 5 * w4;
}

template <class T, int V, bool R = true>
__device__ __forceinline__ void solve_ir_instance(const BatchArgs& a, const BatchEntry& e, SolveCommon c,
                                                  unsigned char* base, ClusterTeam& tm, double* red,
                                                  unsigned char* dsm) {
  const long long W = (long long)tm.size() * (blockDim.x >> 5);
  c.un = make_units(e.nx, e.ny, V, W, a.min_rows);
  const int ldi = ir_ld(e.nx);
  const size_t vr = vec_bytes(e.ny, ldi, sizeof(T));
  const size_t vf = vec_bytes(e.ny, ldi, 4);
  IrArgs<T> s;
  s.c = c;
  s.b = Grid<const double>{static_cast<const double*>(e.b), e.ld};
  s.x = Grid<double>{static_cast<double*>(e.x), e.ld};
  s.r = Grid<T>{reinterpret_cast<T*>(base), ldi};
  s.p0 = Grid<T>{reinterpret_cast<T*>(base + vr), ldi};
  s.p1 = Grid<T>{reinterpret_cast<T*>(base + 2 * vr), ldi};
  s.z = Grid<float>{reinterpret_cast<float*>(base + 3 * vr), ldi};
  s.d = Grid<float>{reinterpret_cast<float*>(base + 3 * vr + vf), ldi};
  s.store_z = a.store_z > 0 ? 1 : 0;
  s.max_outer = a.max_outer;
  // the single solves' inner caps: binary32 4 (nx + ny) + 50, bf16 p, r 2 (nx + ny) + 50
  s.maxit_inner = a.maxit_inner > 0 ? a.maxit_inner : (sizeof(T) == 2 ? 2 : 4) * (e.nx + e.ny) + 50;
  s.tol_inner = a.tol_inner;
  s.uo = make_units(e.nx, e.ny, 2, W, a.min_rows);
  ir_solve<T, V, 2, R>(s, tm, red, dsm);
}

template <int KIND, bool R>
__device__ __forceinline__ void solve_instance(const BatchArgs& a, const BatchEntry& e, ClusterTeam& tm, double* red,
                                               unsigned char* dsm) {
  using T = typename KindTraits<KIND>::T;
  constexpr int V = KindTraits<KIND>::V;
  SolveCommon c;
  c.nx = e.nx;
  c.ny = e.ny;
  c.un = make_units(e.nx, e.ny, V, (long long)tm.size() * (blockDim.x >> 5), a.min_rows);
  c.ctl = nullptr;
  c.info = a.info + e.idx;
  c.history = nullptr;
  c.tol = a.tol;
  c.maxit = a.maxit;
  c.true_res = a.true_res;
  c.timeout_ns = 2000000000LL;
  c.rg = a.rg;
  c.err = a.errs + e.idx;
  c.abort_flag = nullptr;
  unsigned char* base = a.ws + e.ws_off;
  if constexpr (KIND == KIND_F64_CLASSIC || KIND == KIND_F32_CLASSIC) {
    const size_t vb = vec_bytes(e.ny, e.ld, sizeof(T));
    ClassicArgs<T> s;
    s.c = c;
    s.b = Grid<const T>{static_cast<const T*>(e.b), e.ld};
    s.x = Grid<T>{static_cast<T*>(e.x), e.ld};
    s.r = Grid<T>{reinterpret_cast<T*>(base), e.ld};
    s.p0 = Grid<T>{reinterpret_cast<T*>(base + vb), e.ld};
    s.p1 = Grid<T>{reinterpret_cast<T*>(base + 2 * vb), e.ld};
    s.z = Grid<T>{reinterpret_cast<T*>(base + 3 * vb), e.ld};
    s.store_z = a.store_z >= 0 ? a.store_z : (sizeof(T) == 8 ? 1 : 0);
    classic_solve<T, V, R>(s, tm, red, dsm);
  } else if constexpr (KIND == KIND_F64_NEWCG || KIND == KIND_F32_NEWCG) {
    const size_t vb = vec_bytes(e.ny, e.ld, sizeof(T));
    NewcgArgs<T> s;
    s.c = c;
    s.b = Grid<const T>{static_cast<const T*>(e.b), e.ld};
    s.x = Grid<T>{static_cast<T*>(e.x), e.ld};
    s.r = Grid<T>{reinterpret_cast<T*>(base), e.ld};
    s.w0 = Grid<T>{reinterpret_cast<T*>(base + vb), e.ld};
    s.w1 = Grid<T>{reinterpret_cast<T*>(base + 2 * vb), e.ld};
    s.z = Grid<T>{reinterpret_cast<T*>(base + 3 * vb), e.ld};
    s.q = Grid<T>{reinterpret_cast<T*>(base + 4 * vb), e.ld};
    s.p = Grid<T>{reinterpret_cast<T*>(base + 5 * vb), e.ld};
    s.rr_period = a.rr_period;
    newcg_solve<T, V, R>(s, tm, red, dsm);
  } else {
    // inner passes: eight columns a lane (ring kernels) where the wider strip
    // pads the row less than it gains, else four; outer passes: two
    if constexpr (R) {
      if (ir_wide(e.nx)) {
        solve_ir_instance<T, 8>(a, e, c, base, tm, red, dsm);
        return;
      }
    }
    solve_ir_instance<T, 4, R>(a, e, c, base, tm, red, dsm);
  }
}

template <int KIND, bool R>
__global__ void __launch_bounds__(512) k_batched(const BatchArgs a) {
  __shared__ double red[kRedDoubles];
  __shared__ int s_item;
  extern __shared__ __align__(128) unsigned char dsm[];
  ClusterTeam tm{0ull};
  auto cl = cooperative_groups::this_cluster();
  for (;;) {
    if (tm.rank() == 0 && threadIdx.x == 0) s_item = (int)atomicAdd(&a.bctl->next, 1u);
    tm.barrier();
    const int item = *cl.map_shared_rank(&s_item, 0);
    tm.barrier();  // every CTA has read the item before rank 0 fetches the next
    if (item >= a.count) break;
    const BatchEntry e = a.tab[item];
    solve_instance<KIND, R>(a, e, tm, red, dsm);
  }
}

static int kind_of(int variant, int precision) {
  switch (precision) {
    case LAP5CG_PREC_F64: return variant == LAP5CG_NEWCG ? KIND_F64_NEWCG : KIND_F64_CLASSIC;
    case LAP5CG_PREC_F32: return variant == LAP5CG_NEWCG ? KIND_F32_NEWCG : KIND_F32_CLASSIC;
    case LAP5CG_PREC_IR_F32: return variant == LAP5CG_NEWCG ? -1 : KIND_IR_F32;
    case LAP5CG_PREC_IR_BF16PR: return variant == LAP5CG_NEWCG ? -1 : KIND_IR_BF16;
    default: return -1;
  }
}

static const void* kernel_of(int kind, bool ring) {
#define LAP5_K(K) (ring ? reinterpret_cast<const void*>(&k_batched<K, true>) \
                        : reinterpret_cast<const void*>(&k_batched<K, false>))
  switch (kind) {
    case KIND_F64_CLASSIC: return LAP5_K(KIND_F64_CLASSIC);
    case KIND_F64_NEWCG: return LAP5_K(KIND_F64_NEWCG);
    case KIND_F32_CLASSIC: return LAP5_K(KIND_F32_CLASSIC);
    case KIND_F32_NEWCG: return LAP5_K(KIND_F32_NEWCG);
    case KIND_IR_F32: return LAP5_K(KIND_IR_F32);
    default: return LAP5_K(KIND_IR_BF16);
  }
#undef LAP5_K
}

// Lane vector width of a kind (alignment requirement of the caller's rows).
static int kind_vec(int kind) { return (kind == KIND_F64_CLASSIC || kind == KIND_F64_NEWCG) ? 2 : 4; }
static size_t kind_elem(int kind) { return (kind == KIND_F32_CLASSIC || kind == KIND_F32_NEWCG) ? 4 : 8; }

static size_t table_bytes(int count) {
  return align_up((size_t)count * sizeof(BatchEntry), kAlign) + align_up((size_t)count * sizeof(int), kAlign);
}

static int ring_slot_kind(int kind) {
  switch (kind) {
    case KIND_F64_CLASSIC: return ring_slot_classic(2, 8);
    case KIND_F64_NEWCG: return ring_slot_newcg(2, 8);
    case KIND_F32_CLASSIC: return ring_slot_classic(4, 4);
    case KIND_F32_NEWCG: return ring_slot_newcg(4, 4);
    case KIND_IR_F32: return ring_slot_ir(8, 4);  // wide instances take eight columns a lane
    default: return ring_slot_ir(8, 2);
  }
}

size_t batched_ws(int count, const int* nx, const int* ny, const int* ld, int variant, int precision) {
  const int kind = kind_of(variant, precision);
  if (kind < 0 || count < 1 || count > LAP5CG_MAX_BATCH || !nx || !ny || !ld) return 0;
  size_t s = kAlign + table_bytes(count);  // BatchCtl + table
  for (int k = 0; k < count; ++k) {
    if (nx[k] < 1 || ny[k] < 1 || ld[k] < nx[k] || (long long)ny[k] * ld[k] > (1LL << 34)) return 0;
    s += instance_bytes(kind, nx[k], ny[k], ld[k]);
  }
  return s;
}

int solve_batched(int count, const int* nx, const int* ny, const int* ld, const void* const* b, void* const* x,
                  double tol, int maxit, int variant, int precision, void* workspace, size_t ws_bytes,
                  lap5cg_info* info, const lap5cg_opts& o, cudaStream_t st) {
  const int kind = kind_of(variant, precision);
  if (kind < 0) return LAP5CG_ERR_UNSUPPORTED;
  const size_t need = batched_ws(count, nx, ny, ld, variant, precision);
  if (need == 0) return LAP5CG_ERR_INVALID_ARG;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign) || ws_bytes < need) return LAP5CG_ERR_WORKSPACE;
  const int vw = kind_vec(kind);
  const size_t es = kind_elem(kind);
  std::vector<BatchEntry> tab(count);
  std::vector<int> order(count);
  for (int k = 0; k < count; ++k) {
    if (!b[k] || !x[k]) return LAP5CG_ERR_INVALID_ARG;
    if (ld[k] % vw || reinterpret_cast<uintptr_t>(b[k]) % 16 || reinterpret_cast<uintptr_t>(x[k]) % 16)
      return LAP5CG_ERR_INVALID_ARG;  // batched solves need 16-byte aligned rows (no staging)
    const size_t bytes = (size_t)ny[k] * ld[k] * es;
    const uintptr_t b0 = reinterpret_cast<uintptr_t>(b[k]), x0 = reinterpret_cast<uintptr_t>(x[k]);
    if (b0 < x0 + bytes && x0 < b0 + bytes) return LAP5CG_ERR_INVALID_ARG;
    order[k] = k;
  }
  // instances that fit in one cluster's shared memory (F64 / F32): the
  // cluster-resident kernel, one cluster an instance, launched first
  std::vector<char> taken;
  int rc = small_batched(count, nx, ny, ld, b, x, tol, maxit, variant, precision, info, o, st, taken);
  if (rc != LAP5CG_OK) return rc;
  order.erase(std::remove_if(order.begin(), order.end(), [&](int k) { return taken[k] != 0; }), order.end());
  const int nbig = (int)order.size();
  if (nbig == 0) return LAP5CG_OK;
  // largest estimated work first (LPT)
  std::stable_sort(order.begin(), order.end(), [&](int i, int j) {
    const double wi = (double)nx[i] * ny[i] * (nx[i] + ny[i]), wj = (double)nx[j] * ny[j] * (nx[j] + ny[j]);
    return wi > wj;
  });
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  BatchCtl* bctl = reinterpret_cast<BatchCtl*>(ws);
  BatchEntry* dtab = reinterpret_cast<BatchEntry*>(ws + kAlign);
  int* errs = reinterpret_cast<int*>(ws + kAlign + align_up((size_t)count * sizeof(BatchEntry), kAlign));
  const size_t inst0 = kAlign + table_bytes(count);
  size_t off = inst0;
  tab.resize(nbig);
  for (int k = 0; k < nbig; ++k) {
    const int i = order[k];
    tab[k].b = b[i];
    tab[k].x = x[i];
    tab[k].ws_off = (long long)off;
    tab[k].nx = nx[i];
    tab[k].ny = ny[i];
    tab[k].ld = ld[i];
    tab[k].idx = i;
    off += instance_bytes(kind, nx[i], ny[i], ld[i]);
  }
  for (int first = 0; first < nbig; first += kFillChunk) {
    FillArgs fa;
    fa.dst = dtab;
    fa.first = first;
    fa.n = std::min(kFillChunk, nbig - first);
    for (int k = 0; k < fa.n; ++k) fa.e[k] = tab[first + k];
    k_fill_table<<<1, kFillChunk, 0, st>>>(fa);
    if (cudaGetLastError() != cudaSuccess) return LAP5CG_ERR_CUDA;
  }
  if (cudaMemsetAsync(bctl, 0, sizeof(BatchCtl), st) != cudaSuccess) return LAP5CG_ERR_CUDA;
  if (cudaMemsetAsync(errs, 0, (size_t)count * sizeof(int), st) != cudaSuccess) return LAP5CG_ERR_CUDA;  // caller order

  int wpc = o.warps_per_cta > 0 ? o.warps_per_cta : 8;  // batched teams measured best with 8
  if (wpc > 16) wpc = 16;
  BatchArgs a;
  a.errs = errs;
  a.count = nbig;
  a.tab = dtab;
  a.bctl = bctl;
  a.ws = ws;
  a.info = info;
  a.tol = tol;
  a.maxit = maxit;
  a.min_rows = o.min_rows > 0 ? o.min_rows : 8;
  a.true_res = o.true_residual;
  a.store_z = o.store_z;
  a.rr_period = o.rr_period;
  a.max_outer = o.max_outer > 0 ? o.max_outer : 60;
  a.maxit_inner = o.maxit_inner;
  a.tol_inner = o.tol_inner > 0.0 ? o.tol_inner : (kind == KIND_IR_BF16 ? 1e-2 : 1e-4);

  int team = o.team_ctas > 0 ? o.team_ctas : 8;
  if (team != 1 && team != 2 && team != 4 && team != 8 && team != 16) return LAP5CG_ERR_INVALID_ARG;
  size_t dyn = 0;
  const bool auto_on = true;  // as for single solves
  rc = choose_ring(kernel_of(kind, true), ring_slot_kind(kind), o, wpc, &a.rg, &dyn, auto_on);
  if (rc != LAP5CG_OK) return rc;
  if (a.rg.S > 0 && dyn < (size_t)wpc * (size_t)a.rg.warp_bytes) return LAP5CG_ERR_INVALID_ARG;
  const void* fn = kernel_of(kind, a.rg.S > 0);
  if (team > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return LAP5CG_ERR_CUDA;
  cudaLaunchConfig_t lc = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = team;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  lc.blockDim = dim3(32 * wpc);
  lc.dynamicSmemBytes = dyn;
  lc.stream = st;
  lc.attrs = attr;
  lc.numAttrs = 1;
  lc.gridDim = dim3(team);
  int maxclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&maxclusters, fn, &lc) != cudaSuccess || maxclusters < 1)
    return LAP5CG_ERR_UNSUPPORTED;
  int nclusters = o.ctas > 0 ? std::max(1, o.ctas / team) : maxclusters;
  if (nclusters > maxclusters) nclusters = maxclusters;
  if (nclusters > nbig) nclusters = nbig;
  lc.gridDim = dim3(nclusters * team);
  void* args[] = {&a};
  return cudaLaunchKernelExC(&lc, fn, args) == cudaSuccess ? LAP5CG_OK : LAP5CG_ERR_CUDA;
}

}  // namespace lap5
