// launch.h -- host-side launch interface between the C ABI (api.cu) and the
// kernel translation units.  Internal to liblap5cg.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "../../include/lap5cg.h"
#include "ring.cuh"

namespace lap5 {

// Launch geometry chosen on the host.
struct LaunchCfg {
  int ctas;           // persistent CTAs (all co-resident)
  int threads;        // threads per CTA
  size_t dyn_smem;    // dynamic shared memory per CTA (row ring)
  int ns, nseg, seg_rows, nunits;  // warp-unit decomposition
};

// One solve on device buffers that already satisfy the vector-path layout:
// every row 16-byte aligned, ld a multiple of the lane vector width.
struct SolvePlan {
  int nx, ny, ld;              // ld of b and x (user or staged)
  int ldw;                     // ld of workspace vectors
  const void* b;
  void* x;
  unsigned char* ws;           // workspace base (control block first)
  size_t ws_bytes;
  lap5cg_info* info;
  double tol;
  int maxit;
  int variant, precision;
  lap5cg_opts opts;
};

int apply_dispatch(int nx, int ny, int ld, int dtype, const void* x, void* y, cudaStream_t st);

// Workspace layout queries (bytes), per precision family.
size_t ws_bytes_f64(int nx, int ny, int ldw, int variant);
size_t ws_bytes_f32(int nx, int ny, int ldw, int variant);
size_t ws_bytes_ir(int nx, int ny, int variant, int precision);
size_t ws_bytes_mg(int nx, int ny, int ldw, int variant, int precision);

size_t batched_ws(int count, const int* nx, const int* ny, const int* ld, int variant, int precision);
int solve_batched(int count, const int* nx, const int* ny, const int* ld, const void* const* b, void* const* x,
                  double tol, int maxit, int variant, int precision, void* workspace, size_t ws_bytes,
                  lap5cg_info* info, const lap5cg_opts& o, cudaStream_t st);

// Cluster-resident solve of a small grid (F64 / F32): *used = false when the
// grid does not fit or the options ask for the streaming kernels.
int try_small(const SolvePlan& p, cudaStream_t st, bool* used);

// Batched solves: the instances that fit in one cluster's shared memory are
// solved by the cluster-resident kernel (one cluster an instance); taken[k]
// is set for them (count entries).
int small_batched(int count, const int* nx, const int* ny, const int* ld, const void* const* b, void* const* x,
                  double tol, int maxit, int variant, int precision, lap5cg_info* info, const lap5cg_opts& o,
                  cudaStream_t st, std::vector<char>& taken);

int solve_f64(const SolvePlan& p, cudaStream_t st);
int solve_f32(const SolvePlan& p, cudaStream_t st);
int solve_ir(const SolvePlan& p, cudaStream_t st);
int solve_mg(const SolvePlan& p, cudaStream_t st);

// Device properties cached per device.
struct DevProps {
  int sms;
  int max_smem_optin;
};
int dev_props(DevProps* out);

// Grid sizing shared by the persistent kernels: fills cfg from the occupancy
// of kernel func at the requested warps per CTA.
int plan_units(const void* func, int nx, int ny, int V, const lap5cg_opts& o, size_t dyn_smem, LaunchCfg* cfg,
               int row_align = 1);

// Row-ring geometry for a kernel whose largest ring slot is slot_bytes: sets
// the kernel's dynamic shared memory limit and returns the bytes per CTA
// (S = 0 and 0 bytes when the ring is off or does not fit).  auto_on: whether
// ring_slots = 0 (automatic) turns the ring on for this kernel family.
// wpc: the warps per CTA the kernel will be launched with (every warp gets a
// ring of its own in the dynamic shared memory).
int choose_ring(const void* func, int slot_bytes, const lap5cg_opts& o, int wpc, RingGeom* g, size_t* dyn_smem,
                bool auto_on);

// Warps per CTA of the single-grid kernels for these options.
int warps_of(const lap5cg_opts& o);

// Largest ring slot (bytes) of each kernel family, V = lane vector width.
inline int ring_slot_classic(int V, int es) {
  const int M = 32 * V * es;
  const int p = 2 * (M + 32) + M, rz = 2 * M, rr = (M + 32) + 2 * M;  // phase P carries x for the deferred update
  return p > rz ? (p > rr ? p : rr) : (rz > rr ? rz : rr);
}
inline int ring_slot_newcg(int V, int es) { return (32 * V * es + 32) + 5 * 32 * V * es; }
inline int ring_slot_ir(int V, int es_r) {
  const int Mr = 32 * V * es_r, Mf = 32 * V * 4;
  const int p = 2 * (Mr + 32), r = (Mr + 32) + Mf + Mr;
  return p > r ? p : r;
}

// Launch defaults (measured on GB300; the autotuner can override them).
constexpr int kDefaultWarps = 4;          // warps per CTA
constexpr int kDefaultMinRows = 2;        // shortest warp unit (rows) on small grids
constexpr int kRingBytesPerWarp = 12800;  // 16 warps per SM fit 228 KB of shared memory
constexpr int kRingMinRows = 8;           // automatic ring only for units at least this tall

constexpr size_t kCtlBytes = 256 * 1024;  // control block region at the workspace start
constexpr size_t kAlign = 256;
__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace lap5
