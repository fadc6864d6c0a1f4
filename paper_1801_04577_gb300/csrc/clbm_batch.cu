// Batched solves of many independent lattices (declarations in include/clbm.h).
//
// All lattices live in one arena (two ping-pong buffers); each lattice is also
// an ordinary clbm_ctx "view" over its slice of the arena, so boundaries,
// initialisation, moments and Nusselt numbers reuse the single-lattice code.
// A solve replays one CUDA graph per K steps: K launches (per launch group)
// of the tile-list step kernel, the per-lattice residual, and three small
// kernels that retire converged lattices and rebuild the tile lists on the
// device.  The host only reads back the active count after each replay.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/clbm.h"
#include "clbm_internal.h"

using namespace clbm;

namespace {

constexpr int kWidthChoices[kBatchGroups] = {1, 2, 4};  // nodes per lane; a warp covers 32 x this

int group_id(int v) { return v == 1 ? 0 : (v == 2 ? 1 : 2); }

int width_class(int nx) { return nx <= 48 ? 0 : (nx <= 96 ? 1 : (nx <= 192 ? 2 : 3)); }

__global__ void batch_update_kernel(int n, int* __restrict__ active, const double* __restrict__ res,
                                    double tol, long long* __restrict__ conv, BatchCtl* ctl, int K) {
  __shared__ int nact;
  __shared__ long long t;
  if (threadIdx.x == 0) {
    ctl->t += K;
    t = ctl->t;
    nact = 0;
  }
  __syncthreads();
  int local = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (!active[i]) continue;
    const double r = res[i];
    if (!isfinite(r)) {  // diverged: retire and flag
      active[i] = 0;
      conv[i] = -2;
    } else if (r < tol) {
      active[i] = 0;
      conv[i] = t;
    } else {
      ++local;
    }
  }
  atomicAdd(&nact, local);
  __syncthreads();
  if (threadIdx.x == 0) ctl->n_active = nact;
}

// Offsets of each active lattice's tiles inside its group (serial: n is small).
__global__ void batch_scan_kernel(int n, const int* __restrict__ active,
                                  const int* __restrict__ group_of, const int* __restrict__ tiles_of,
                                  long long* __restrict__ offset, BatchCtl* ctl) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  long long cnt[kBatchGroups];
  for (int g = 0; g < kBatchGroups; ++g) cnt[g] = 0;
  int nact = 0;
  for (int i = 0; i < n; ++i) {
    if (!active[i]) {
      offset[i] = -1;
      continue;
    }
    ++nact;
    const int g = group_of[i];
    offset[i] = cnt[g];
    cnt[g] += tiles_of[i];
  }
  for (int g = 0; g < kBatchGroups; ++g) ctl->count[g] = (int)cnt[g];
  ctl->n_active = nact;
}

// Tiles {lattice, row, first x, 0} of rows y0 .. y0 + rows - 1 (the rows that
// are not boundary rows) of every active lattice.
__global__ void batch_tiles_kernel(int n, const int* __restrict__ active,
                                   const long long* __restrict__ offset,
                                   const int* __restrict__ group_of, const int* __restrict__ rows_of,
                                   const int* __restrict__ tpr_of, const int* __restrict__ width_of,
                                   const int* __restrict__ y0_of, int4* const* __restrict__ group_tiles) {
  const int i = blockIdx.x;
  if (i >= n || !active[i]) return;
  int4* dst = group_tiles[group_of[i]] + offset[i];
  const int tpr = tpr_of[i], w = width_of[i], y0 = y0_of[i];
  const int total = rows_of[i] * tpr;
  for (int k = threadIdx.x; k < total; k += blockDim.x)
    dst[k] = make_int4(i, y0 + k / tpr, (k % tpr) * w, 0);
}

}  // namespace

struct clbm_batch {
  int n = 0;
  int precision = 0, rounding = 0;
  const Launchers* L = nullptr;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* arena[2] = {nullptr, nullptr};
  std::vector<clbm_ctx*> views;
  std::vector<int> nx, ny, py, masked, width, group;
  std::vector<long long> nodes;
  std::vector<int> grid;  // per group
  std::vector<long long> group_base = std::vector<long long>(kBatchGroups, 0);  // tile-list offsets
  BatchLat* d_lats = nullptr;
  int* d_active = nullptr;
  double* d_res = nullptr;
  long long* d_conv = nullptr;
  BatchCtl* d_ctl = nullptr;
  BatchCtl* h_ctl = nullptr;  // pinned
  long long* d_offset = nullptr;
  int* d_ints = nullptr;  // group_of, tiles_of, rows_of, tpr_of, width_of, y0_of (6 x n)
  int4* d_tiles = nullptr;
  long long tile_cap = 0;
  int4** d_group_tiles = nullptr;
  double* d_snap = nullptr;  // convergence snapshots of all lattices
  int* d_snap_valid = nullptr;
  int2* d_bent = nullptr;  // boundary entries {lattice, node} of all lattices
  int nbent = 0;
  double* d_rpart = nullptr;  // residual chunk sums
  int res_chunks = 1;
  cudaGraphExec_t exec = nullptr;
  int exec_K = 0;
  double exec_tol = -1.0;
  std::string err;
};

static clbm_status bfail(clbm_batch* b, clbm_status s, const std::string& m) {
  if (b) b->err = m;
  return s;
}

#define BCUDA(b, call)                                                                        \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return bfail((b), CLBM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Rows that get interior tiles: all rows of a periodic y axis, else all but the
// first and last (boundary rows).
static int interior_rows(const clbm_batch* b, int i) {
  return b->py[i] ? b->ny[i] : std::max(b->ny[i] - 2, 0);
}

// Upload the per-lattice launch layout (group, tile counts) for the current widths.
static clbm_status upload_layout(clbm_batch* b, const std::vector<int>& active) {
  const int n = b->n;
  std::vector<int> ints(6 * (size_t)n);
  std::vector<long long> gcap(kBatchGroups, 0);
  for (int i = 0; i < n; ++i) {
    const int w = 32 * b->width[i];
    const int tpr = (b->nx[i] + w - 1) / w;
    const int rows = interior_rows(b, i);
    b->group[i] = group_id(b->width[i]);
    ints[i] = b->group[i];
    ints[n + i] = rows * tpr;
    ints[2 * n + i] = rows;
    ints[3 * n + i] = tpr;
    ints[4 * n + i] = w;
    ints[5 * n + i] = b->py[i] ? 0 : 1;
    gcap[b->group[i]] += (long long)rows * tpr;
  }
  std::vector<int4*> bases(kBatchGroups);
  long long off = 0;
  for (int g = 0; g < kBatchGroups; ++g) {
    b->group_base[g] = off;
    bases[g] = b->d_tiles + off;
    off += gcap[g];
  }
  if (off > b->tile_cap) return bfail(b, CLBM_EINVAL, "tile list exceeds its capacity");
  BCUDA(b, cudaMemcpyAsync(b->d_ints, ints.data(), ints.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
  BCUDA(b, cudaMemcpyAsync(b->d_group_tiles, bases.data(), kBatchGroups * sizeof(int4*), cudaMemcpyHostToDevice, b->stream));
  BCUDA(b, cudaMemcpyAsync(b->d_active, active.data(), n * sizeof(int), cudaMemcpyHostToDevice, b->stream));
  BCUDA(b, cudaStreamSynchronize(b->stream));
  return CLBM_OK;
}

static clbm_status build_tiles(clbm_batch* b) {
  const int n = b->n;
  const int* gi = b->d_ints;
  batch_scan_kernel<<<1, 32, 0, b->stream>>>(n, b->d_active, gi, gi + n, b->d_offset, b->d_ctl);
  BCUDA(b, cudaGetLastError());
  batch_tiles_kernel<<<n, 256, 0, b->stream>>>(n, b->d_active, b->d_offset, gi, gi + 2 * n, gi + 3 * n,
                                               gi + 4 * n, gi + 5 * n, b->d_group_tiles);
  BCUDA(b, cudaGetLastError());
  return CLBM_OK;
}

// One step of every active lattice; parity = which buffer holds the current state.
// Interior tiles first (one launch per tile-width group), then the boundary nodes
// (which, next to solids, replace the provisional values the tiles wrote).
static clbm_status launch_steps(clbm_batch* b, int parity, int tstep) {
  std::vector<int> used(kBatchGroups, 0);
  for (int i = 0; i < b->n; ++i) used[b->group[i]] = 1;
  const std::vector<long long>& base = b->group_base;  // as in upload_layout
  for (int g = 0; g < kBatchGroups; ++g) {
    if (!used[g]) continue;
    const int v = kWidthChoices[g];
    if (b->grid[g] <= 0) return bfail(b, CLBM_ECUDA, "no occupancy for the batched step kernel");
    BCUDA(b, b->L->batch_step(v, b->d_lats, b->d_tiles + base[g], &b->d_ctl->count[g], parity,
                              &b->d_ctl->t, tstep, b->rounding, b->grid[g], b->stream));
  }
  BCUDA(b, b->L->batch_boundary(b->d_lats, b->d_bent, b->nbent, b->d_active, parity, &b->d_ctl->t,
                                tstep, b->rounding, b->stream));
  return CLBM_OK;
}

static void release(clbm_batch* b) {
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (clbm_ctx* v : b->views) clbm_destroy(v);
  b->views.clear();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  cudaFree(b->arena[0]);
  cudaFree(b->arena[1]);
  cudaFree(b->d_lats);
  cudaFree(b->d_active);
  cudaFree(b->d_res);
  cudaFree(b->d_conv);
  cudaFree(b->d_ctl);
  cudaFree(b->d_offset);
  cudaFree(b->d_ints);
  cudaFree(b->d_tiles);
  cudaFree(b->d_group_tiles);
  cudaFree(b->d_bent);
  cudaFree(b->d_rpart);
  cudaFree(b->d_snap);
  cudaFree(b->d_snap_valid);
  if (b->h_ctl) cudaFreeHost(b->h_ctl);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

static clbm_status init_all(clbm_batch* b, const clbm_batch_item* items) {
  for (int i = 0; i < b->n; ++i) {
    const clbm_batch_item& it = items[i];
    clbm_status st = clbm_init_fields(b->views[i], it.rho, it.ux, it.uy, it.T, 0);
    if (st != CLBM_OK) return bfail(b, st, "lattice " + std::to_string(i) + ": " + clbm_last_error(b->views[i]));
  }
  return CLBM_OK;
}

// Pick the tile width per class of row length by timing the batched step.
static clbm_status autotune(clbm_batch* b) {
  const int n = b->n;
  const int nchoice = b->L->vec >= 4 ? 3 : 2;
  std::vector<int> best(4, b->L->vec);
  cudaEvent_t e0, e1;
  BCUDA(b, cudaEventCreate(&e0));
  BCUDA(b, cudaEventCreate(&e1));
  for (int cls = 0; cls < 4; ++cls) {
    std::vector<int> active(n, 0);
    long long nodes = 0;
    for (int i = 0; i < n; ++i)
      if (width_class(b->nx[i]) == cls) {
        active[i] = 1;
        nodes += b->nodes[i];
      }
    if (nodes == 0) continue;
    float best_t = 1e30f;
    for (int c = 0; c < nchoice; ++c) {
      for (int i = 0; i < n; ++i)
        if (active[i]) b->width[i] = kWidthChoices[c];
      clbm_status st = upload_layout(b, active);
      if (st != CLBM_OK) return st;
      if ((st = build_tiles(b)) != CLBM_OK) return st;
      for (int k = 0; k < 2; ++k)
        if ((st = launch_steps(b, k & 1, k)) != CLBM_OK) return st;
      BCUDA(b, cudaEventRecord(e0, b->stream));
      for (int k = 0; k < 6; ++k)
        if ((st = launch_steps(b, k & 1, k)) != CLBM_OK) return st;
      BCUDA(b, cudaEventRecord(e1, b->stream));
      BCUDA(b, cudaEventSynchronize(e1));
      float ms = 0;
      BCUDA(b, cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_t) {
        best_t = ms;
        best[cls] = kWidthChoices[c];
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int i = 0; i < n; ++i) b->width[i] = best[width_class(b->nx[i])];
  return CLBM_OK;
}

extern "C" {

const char* clbm_batch_last_error(const clbm_batch* b) { return b ? b->err.c_str() : ""; }

clbm_status clbm_batch_destroy(clbm_batch* b) {
  if (!b) return CLBM_OK;
  release(b);
  delete b;
  return CLBM_OK;
}

clbm_status clbm_batch_create(const clbm_batch_item* items, int32_t n, int32_t autotune_tiles,
                              void* stream, clbm_batch** out) {
  if (!out) return CLBM_EINVAL;
  *out = nullptr;
  if (!items || n < 1) return CLBM_EINVAL;
  const int prec = items[0].params.precision, rnd = items[0].params.rounding;
  const Launchers* L = prec == CLBM_F64 ? &kLaunchF64 : prec == CLBM_F32 ? &kLaunchF32
                     : prec == CLBM_F16DEV ? &kLaunchF16 : prec == CLBM_BF16DEV ? &kLaunchBF16 : nullptr;
  if (!L) return CLBM_EINVAL;
  for (int i = 0; i < n; ++i)
    if (items[i].params.precision != prec || items[i].params.rounding != rnd ||
        items[i].params.viscous_heating != 0)
      return CLBM_EINVAL;
  clbm_batch* b = new (std::nothrow) clbm_batch();
  if (!b) return CLBM_ENOMEM;
  b->n = n;
  b->precision = prec;
  b->rounding = rnd;
  b->L = L;
  b->grid.assign(kBatchGroups, 0);
  auto bail = [&](clbm_status st) {
    release(b);
    delete b;
    return st;
  };
  if (stream) {
    b->stream = static_cast<cudaStream_t>(stream);
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(CLBM_ECUDA);
    b->own_stream = true;
  }
  // arena layout
  std::vector<size_t> off(n);
  size_t total = 0;
  for (int i = 0; i < n; ++i) {
    const clbm_params& p = items[i].params;
    if (p.nx < 1 || p.ny < 1 || p.ny > 65535) return bail(CLBM_EINVAL);
    off[i] = total;
    total += (view_buffer_bytes(p.nx, p.ny, prec, 0) + 255) / 256 * 256;
  }
  for (int k = 0; k < 2; ++k)
    if (cudaMalloc(&b->arena[k], total) != cudaSuccess) {
      cudaGetLastError();
      return bail(CLBM_ENOMEM);
    }
  b->views.assign(n, nullptr);
  long long cap = 0;
  for (int i = 0; i < n; ++i) {
    const clbm_batch_item& it = items[i];
    clbm_status st = create_view(&it.params, b->stream, static_cast<char*>(b->arena[0]) + off[i],
                                 static_cast<char*>(b->arena[1]) + off[i], &b->views[i]);
    if (st != CLBM_OK) return bail(st);
    st = clbm_set_boundaries(b->views[i], it.solid, it.tbc, it.n_tbc, it.side_tbc, it.links, it.n_links);
    if (st != CLBM_OK) return bail(st);
    b->nx.push_back(it.params.nx);
    b->ny.push_back(it.params.ny);
    b->py.push_back(it.params.periodic_y ? 1 : 0);
    b->nodes.push_back((long long)it.params.nx * it.params.ny);
    cap += (long long)it.params.ny * ((it.params.nx + 31) / 32);
  }
  if (cap >= (1LL << 31)) return bail(CLBM_EINVAL);
  // device tables
  long long snap_total = 0;
  for (int i = 0; i < n; ++i) snap_total += 3 * b->nodes[i];
  if (cudaMalloc(&b->d_snap, snap_total * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&b->d_snap_valid, n * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return bail(CLBM_ENOMEM);
  }
  std::vector<BatchLat> lats(n);
  std::vector<int2> bent;
  long long snap_off = 0;
  b->masked.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    const ViewInfo v = describe_view(b->views[i]);
    lats[i].g = v.g;
    lats[i].c = v.c;
    lats[i].buf[0] = v.buf[0];
    lats[i].buf[1] = v.buf[1];
    lats[i].snap = b->d_snap + snap_off;
    snap_off += 3 * b->nodes[i];
    b->masked[i] = v.g.flags != nullptr;
    for (int k = 0; k < v.nb; ++k) bent.push_back(make_int2(i, v.bnodes_host[k]));
  }
  b->nbent = (int)bent.size();
  if (!bent.empty()) {
    if (cudaMalloc(&b->d_bent, bent.size() * sizeof(int2)) != cudaSuccess ||
        cudaMemcpy(b->d_bent, bent.data(), bent.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      return bail(CLBM_ENOMEM);
    }
  }
  b->width.assign(n, L->vec);
  b->group.assign(n, 0);
  b->tile_cap = cap;
  if (cudaMalloc(&b->d_lats, n * sizeof(BatchLat)) != cudaSuccess ||
      cudaMalloc(&b->d_active, n * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&b->d_res, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&b->d_conv, n * sizeof(long long)) != cudaSuccess ||
      cudaMalloc(&b->d_ctl, sizeof(BatchCtl)) != cudaSuccess ||
      cudaMalloc(&b->d_offset, n * sizeof(long long)) != cudaSuccess ||
      cudaMalloc(&b->d_ints, 6 * (size_t)n * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&b->d_tiles, std::max<long long>(cap, 1) * sizeof(int4)) != cudaSuccess ||
      cudaMalloc(&b->d_group_tiles, kBatchGroups * sizeof(int4*)) != cudaSuccess ||
      cudaMallocHost(&b->h_ctl, sizeof(BatchCtl)) != cudaSuccess) {
    cudaGetLastError();
    return bail(CLBM_ENOMEM);
  }
  long long maxnodes = 1;
  for (int i = 0; i < n; ++i) maxnodes = std::max(maxnodes, b->nodes[i]);
  b->res_chunks = (int)((maxnodes + L->residual_chunk - 1) / L->residual_chunk);
  if (cudaMalloc(&b->d_rpart, (size_t)n * b->res_chunks * 8 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return bail(CLBM_ENOMEM);
  }
  if (cudaMemcpy(b->d_lats, lats.data(), n * sizeof(BatchLat), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(b->d_ctl, 0, sizeof(BatchCtl)) != cudaSuccess)
    return bail(CLBM_ECUDA);
  for (int g = 0; g < kBatchGroups; ++g)
    b->grid[g] = kWidthChoices[g] > L->vec ? 0 : L->batch_grid(kWidthChoices[g]);
  if (autotune_tiles) {
    clbm_status st = autotune(b);
    if (st != CLBM_OK) return bail(st);
  }
  clbm_status st = init_all(b, items);
  if (st != CLBM_OK) return bail(st);
  std::vector<int> all(n, 1);
  if ((st = upload_layout(b, all)) != CLBM_OK) return bail(st);
  *out = b;
  return CLBM_OK;
}

clbm_status clbm_batch_damp_period2(clbm_batch* b) {
  if (!b) return CLBM_EINVAL;
  for (int i = 0; i < b->n; ++i) {
    clbm_status st = clbm_damp_period2(b->views[i]);
    if (st != CLBM_OK) return bfail(b, st, "lattice " + std::to_string(i) + ": " + clbm_last_error(b->views[i]));
  }
  BCUDA(b, cudaStreamSynchronize(b->stream));
  return CLBM_OK;
}

clbm_status clbm_batch_tile_width(const clbm_batch* b, int32_t i, int32_t* nodes_per_warp) {
  if (!b || !nodes_per_warp || i < 0 || i >= b->n) return CLBM_EINVAL;
  *nodes_per_warp = 32 * b->width[i];
  return CLBM_OK;
}

clbm_status clbm_batch_lattice(clbm_batch* b, int32_t i, clbm_ctx** view) {
  if (!b || !view || i < 0 || i >= b->n) return CLBM_EINVAL;
  *view = b->views[i];
  return CLBM_OK;
}

clbm_status clbm_batch_solve(clbm_batch* b, double tol, int64_t max_steps, int32_t check_every,
                             int64_t* conv_steps, double* residuals, int64_t* steps_run) {
  if (!b || max_steps < 1 || check_every < 1 || !(tol >= 0)) return bfail(b, CLBM_EINVAL, "bad solve arguments");
  const int n = b->n;
  const int K = (check_every + 1) / 2 * 2;  // even: each replay starts and ends in buffer 0
  // start: every lattice active, counters reset, tile lists rebuilt
  std::vector<int> all(n, 1);
  clbm_status st = upload_layout(b, all);
  if (st != CLBM_OK) return st;
  std::vector<long long> minus1(n, -1);
  BCUDA(b, cudaMemcpyAsync(b->d_conv, minus1.data(), n * sizeof(long long), cudaMemcpyHostToDevice, b->stream));
  BCUDA(b, cudaMemsetAsync(b->d_ctl, 0, sizeof(BatchCtl), b->stream));
  BCUDA(b, cudaMemsetAsync(b->d_snap_valid, 0, n * sizeof(int), b->stream));
  for (int i = 0; i < n; ++i) set_view_time(b->views[i], 0, 0);
  if ((st = build_tiles(b)) != CLBM_OK) return st;
  if (!b->exec || b->exec_K != K || b->exec_tol != tol) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    cudaGraph_t graph;
    BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    clbm_status cst = CLBM_OK;
    for (int j = 0; j < K && cst == CLBM_OK; ++j) cst = launch_steps(b, j & 1, j);
    if (cst == CLBM_OK && b->L->batch_residual(b->d_lats, b->d_active, b->d_snap_valid, b->d_res, n, K,
                                               b->d_rpart, b->res_chunks, b->stream) != cudaSuccess)
      cst = CLBM_ECUDA;
    if (cst == CLBM_OK) {
      batch_update_kernel<<<1, 256, 0, b->stream>>>(n, b->d_active, b->d_res, tol, b->d_conv, b->d_ctl, K);
      const int* gi = b->d_ints;
      batch_scan_kernel<<<1, 32, 0, b->stream>>>(n, b->d_active, gi, gi + n, b->d_offset, b->d_ctl);
      batch_tiles_kernel<<<n, 256, 0, b->stream>>>(n, b->d_active, b->d_offset, gi, gi + 2 * n,
                                                   gi + 3 * n, gi + 4 * n, gi + 5 * n, b->d_group_tiles);
      if (cudaGetLastError() != cudaSuccess) cst = CLBM_ECUDA;
      if (cst == CLBM_OK &&
          cudaMemcpyAsync(b->h_ctl, b->d_ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
        cst = CLBM_ECUDA;
    }
    cudaError_t ee = cudaStreamEndCapture(b->stream, &graph);
    if (cst != CLBM_OK || ee != cudaSuccess) {
      if (ee == cudaSuccess) cudaGraphDestroy(graph);
      cudaGetLastError();
      return bfail(b, CLBM_ECUDA, "graph capture of the batched solve failed");
    }
    ee = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ee != cudaSuccess) return bfail(b, CLBM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ee));
    b->exec_K = K;
    b->exec_tol = tol;  // the tolerance is an argument of the captured update kernel
  }
  b->h_ctl->n_active = n;
  b->h_ctl->t = 0;
  long long t = 0;
  while (true) {
    BCUDA(b, cudaGraphLaunch(b->exec, b->stream));
    BCUDA(b, cudaStreamSynchronize(b->stream));
    t = b->h_ctl->t;
    if (b->h_ctl->n_active == 0 || t >= max_steps) break;
  }
  std::vector<long long> conv(n);
  std::vector<double> res(n);
  BCUDA(b, cudaMemcpy(conv.data(), b->d_conv, n * sizeof(long long), cudaMemcpyDeviceToHost));
  BCUDA(b, cudaMemcpy(res.data(), b->d_res, n * sizeof(double), cudaMemcpyDeviceToHost));
  for (int i = 0; i < n; ++i) {
    if (conv_steps) conv_steps[i] = conv[i];
    if (residuals) residuals[i] = res[i];
    set_view_time(b->views[i], conv[i] > 0 ? conv[i] : t, 0);
  }
  if (steps_run) *steps_run = t;
  return CLBM_OK;
}

}  // extern "C"
