// C ABI of the GB300 cascaded thermal LBM library (declarations and the
// contract of every entry point are in include/clbm.h).
//
// This file holds host code only: argument validation, device memory
// ownership, the boundary description (flags / link tables built once on the
// host), and the launches.  The kernels live in clbm_kernels.cuh and are
// instantiated per storage type in clbm_kernels_*.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/clbm.h"
#include "clbm_internal.h"

using namespace clbm;

namespace {

constexpr int kEX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
constexpr int kEY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
constexpr int kOpp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
constexpr int kMaxRedBlocks = 1024;
// Step graphs: level l holds 2^(l+1) steps, l = 0 .. kGraphLevels - 1 (2 .. 32 steps).
constexpr int kGraphLevels = 5;
constexpr int kGraphSteps = 1 << kGraphLevels;

}  // namespace

struct clbm_ctx {
  clbm_params p{};
  double s3 = 0, l2 = 0;
  const Launchers* L = nullptr;
  int pitch = 0;
  long long plane = 0;
  size_t buf_bytes = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* buf[2] = {nullptr, nullptr};
  bool borrowed = false;  // buffers owned by a batch arena
  // y-slab of a larger lattice: p.ny = stored rows (own rows + one ghost row on
  // each side), p.periodic_y = 0; gny / gpy describe the whole lattice and the
  // own rows [ylo, yhi) hold its rows y0 .. y0 + (yhi - ylo) - 1
  bool slab = false;
  int gny = 0, gpy = 0, y0 = 0;
  int ylo = 0, yhi = 0, ywlo = 0, ywhi = 0;
  cudaEvent_t ev_halo[2] = {nullptr, nullptr};  // orders halo copies between two streams
  int cur = 0;
  int64_t t = 0;
  bool have_walls = false;
  // masked-lattice tables
  uint16_t* d_flags = nullptr;
  int32_t* d_slot = nullptr;
  double* d_lk_ne = nullptr;
  int32_t* d_lk_tbc = nullptr;
  double* d_lk_q = nullptr;
  uint8_t* d_tile_fluid = nullptr;  // masked lattices: which interior warp tiles hold fluid
  int tiles_per_row = 0;
  double* d_tbc = nullptr;
  std::vector<int32_t> h_bnodes;  // nodes the boundary kernel recomputes (pitch layout)
  int32_t* d_bnodes = nullptr;
  std::vector<uint8_t> h_solid;    // [p.ny][nx] over the stored rows (empty: no mask)
  std::vector<clbm_tbc> h_tbc;
  std::vector<clbm_link> h_links;  // links of own-row nodes, node = stored row * nx + x
  int side_tbc[4] = {-1, -1, -1, -1};
  double side_b[4][3] = {};
  double side_u[4][2] = {};  // moving box sides (clbm_set_wall_velocity)
  // scratch
  double* d_fields = nullptr;  // 4 * nx * ny doubles, allocated on first use
  double* d_part = nullptr;    // reduction partials + result
  std::map<int, std::pair<NuLink*, int>> nu_lists;
  // captured step graphs of 2, 4, ..., kGraphSteps steps, keyed by (current buffer, step parity)
  long long* d_t = nullptr;
  cudaGraphExec_t step_graph[4][kGraphLevels] = {};
  std::string err;
};

static void drop_graphs(clbm_ctx* c) {
  for (auto& key : c->step_graph)
    for (auto& g : key)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
}

static clbm_status fail(clbm_ctx* c, clbm_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

static clbm_status cuda_fail(clbm_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  if (c) c->err = m;
  return CLBM_ECUDA;
}

#define CLBM_CUDA(ctx, call)                                   \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call); \
  } while (0)

static const Launchers* launchers_for(int prec) {
  switch (prec) {
    case CLBM_F64: return &kLaunchF64;
    case CLBM_F32: return &kLaunchF32;
    case CLBM_F16DEV: return &kLaunchF16;
    case CLBM_BF16DEV: return &kLaunchBF16;
    default: return nullptr;
  }
}

static DevGeom make_geom(const clbm_ctx* c) {
  DevGeom g;
  g.nx = c->p.nx;
  g.ny = c->p.ny;
  g.pitch = c->pitch;
  g.px = c->p.periodic_x ? 1 : 0;
  g.py = c->p.periodic_y ? 1 : 0;
  g.ylo = c->ylo;
  g.yhi = c->yhi;
  g.ywlo = c->ywlo;
  g.ywhi = c->ywhi;
  g.yoff = c->slab ? c->y0 - 1 : 0;
  g.plane = c->plane;
  g.flags = c->d_flags;
  g.slot = c->d_slot;
  g.lk_ne = c->d_lk_ne;
  g.lk_tbc = c->d_lk_tbc;
  g.lk_q = c->d_lk_q;
  g.tile_fluid = c->d_tile_fluid;
  g.tiles_per_row = c->tiles_per_row;
  g.pad_tiles = 0;
  g.tbc = c->d_tbc;
  std::memcpy(g.side_b, c->side_b, sizeof(g.side_b));
  for (int sd = 0; sd < 4; ++sd)
    for (int k = 0; k < 3; ++k) g.side_bf[sd][k] = (float)c->side_b[sd][k];
  g.moving = 0;
  g.pad_moving = 0;
  for (int sd = 0; sd < 4; ++sd)
    for (int k = 0; k < 2; ++k) {
      g.side_u[sd][k] = c->side_u[sd][k];
      g.side_uf[sd][k] = (float)c->side_u[sd][k];
      if (c->side_u[sd][k] != 0.0) g.moving = 1;
    }
  return g;
}

static DevCoef make_coef(const clbm_ctx* c) {
  DevCoef k;
  k.s_nu = c->p.s_nu;
  k.s_b = c->p.s_b;
  k.s3 = c->s3;
  k.s4 = c->p.s_4;
  k.l0 = c->p.lambda0;
  k.l1 = c->p.lambda1;
  k.l2 = c->l2;
  k.rho0 = c->p.rho0;
  k.T0 = c->p.T0;
  k.gbeta = c->p.gbeta;
  k.Fvx = c->p.Fvx;
  k.Fvy = c->p.Fvy;
  k.Q = c->p.Q;
  k.cT2 = c->p.cT2;
  k.vh = c->p.viscous_heating ? 1 : 0;
  k.pad = 0;
  fill_f32(k);
  return k;
}

static void free_tables(clbm_ctx* c) {
  cudaFree(c->d_flags);
  cudaFree(c->d_slot);
  cudaFree(c->d_lk_ne);
  cudaFree(c->d_lk_tbc);
  cudaFree(c->d_lk_q);
  cudaFree(c->d_tile_fluid);
  cudaFree(c->d_tbc);
  cudaFree(c->d_bnodes);
  c->d_bnodes = nullptr;
  c->d_flags = nullptr;
  c->d_slot = nullptr;
  c->d_lk_ne = nullptr;
  c->d_lk_tbc = nullptr;
  c->d_lk_q = nullptr;
  c->d_tile_fluid = nullptr;
  c->tiles_per_row = 0;
  c->d_tbc = nullptr;
  for (auto& kv : c->nu_lists) cudaFree(kv.second.first);
  c->nu_lists.clear();
}

// Nodes that the interior kernel cannot update on its own: the first and last
// column (walls or the periodic seam), the first and last row of a non-periodic
// y axis, and (masked lattices) every fluid node with a wall or solid among
// its pull sources.  Solid nodes are never listed.
static cudaError_t upload_boundary_list(clbm_ctx* c, const std::vector<uint16_t>& flags) {
  const int nx = c->p.nx;
  std::vector<int32_t>& v = c->h_bnodes;
  v.clear();
  for (int y = c->ylo; y < c->yhi; ++y) {  // own rows only (ghost rows are never updated)
    const bool yedge = (c->ywlo && y == c->ylo) || (c->ywhi && y == c->yhi - 1);
    for (int x = 0; x < nx; ++x) {
      const size_t ip = (size_t)y * c->pitch + x;
      bool need = yedge || x == 0 || x == nx - 1;
      if (!flags.empty()) {
        if (flags[ip] & kFlagSolid) continue;
        need = need || (flags[ip] & 0xFFu);
      }
      if (need) v.push_back((int32_t)ip);
    }
  }
  cudaFree(c->d_bnodes);
  c->d_bnodes = nullptr;
  if (v.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc(&c->d_bnodes, v.size() * sizeof(int32_t));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(c->d_bnodes, v.data(), v.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
}

extern "C" {

const char* clbm_status_string(clbm_status s) {
  switch (s) {
    case CLBM_OK: return "CLBM_OK";
    case CLBM_EINVAL: return "CLBM_EINVAL";
    case CLBM_ENOMEM: return "CLBM_ENOMEM";
    case CLBM_ECUDA: return "CLBM_ECUDA";
    case CLBM_EUNSTABLE: return "CLBM_EUNSTABLE";
    case CLBM_ETIMEOUT: return "CLBM_ETIMEOUT";
    case CLBM_ENOTCONV: return "CLBM_ENOTCONV";
  }
  return "CLBM_UNKNOWN";
}

const char* clbm_last_error(const clbm_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

clbm_status clbm_destroy(clbm_ctx* c) {
  if (!c) return CLBM_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  cudaFree(c->d_t);
  free_tables(c);
  if (!c->borrowed) {
    cudaFree(c->buf[0]);
    cudaFree(c->buf[1]);
  }
  cudaFree(c->d_fields);
  cudaFree(c->d_part);
  for (auto& e : c->ev_halo)
    if (e) cudaEventDestroy(e);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
  return CLBM_OK;
}

// A y-slab: rows [y0, y0 + rows) of the lattice `params` describes.
struct SlabSpec {
  int y0, rows;
};

static clbm_status create_impl(const clbm_params* params, void* stream, void* buf_a, void* buf_b,
                               clbm_ctx** out, const SlabSpec* slab = nullptr) {
  if (!out) return CLBM_EINVAL;
  *out = nullptr;
  if (!params) return CLBM_EINVAL;
  clbm_params pl = *params;
  if (slab) {  // store the own rows plus a ghost row on each side
    if (pl.ny < 1 || slab->rows < 1 || slab->y0 < 0 || (long long)slab->y0 + slab->rows > pl.ny)
      return CLBM_EINVAL;
    pl.ny = slab->rows + 2;
    pl.periodic_y = 0;
  }
  const clbm_params& p = pl;
  const Launchers* L = launchers_for(p.precision);
  if (!L) return CLBM_EINVAL;
  if (p.nx < 1 || p.ny < 1 || p.ny > 65535 || (long long)p.nx * p.ny > (1LL << 31))
    return CLBM_EINVAL;
  auto rate_ok = [](double s) { return std::isfinite(s) && s > 0.0 && s < 2.0; };
  if (p.rounding != 0 && p.rounding != 1) return CLBM_EINVAL;
  if (p.viscous_heating != 0 && p.viscous_heating != 1) return CLBM_EINVAL;
  if (!rate_ok(p.s_nu) || !rate_ok(p.s_b) || !rate_ok(p.s_4) || !rate_ok(p.lambda1) ||
      !(std::isfinite(p.lambda0)) || !(p.rho0 > 0) || !(p.cT2 > 0 && p.cT2 < 0.5))
    return CLBM_EINVAL;
  clbm_ctx* c = new (std::nothrow) clbm_ctx();
  if (!c) return CLBM_ENOMEM;
  c->p = p;
  if (slab) {
    c->slab = true;
    c->gny = params->ny;
    c->gpy = params->periodic_y ? 1 : 0;
    c->y0 = slab->y0;
    c->ylo = 1;
    c->yhi = 1 + slab->rows;
    c->ywlo = !c->gpy && slab->y0 == 0;
    c->ywhi = !c->gpy && slab->y0 + slab->rows == params->ny;
  } else {
    c->gny = p.ny;
    c->gpy = p.periodic_y ? 1 : 0;
    c->ylo = 0;
    c->yhi = p.ny;
    c->ywlo = c->ywhi = p.periodic_y ? 0 : 1;
  }
  c->s3 = p.s_3 > 0 ? p.s_3 : (16.0 - 8.0 * p.s_nu) / (8.0 - p.s_nu);
  c->l2 = p.lambda2 > 0 ? p.lambda2 : 12.0 * (p.lambda1 - 2.0) / (p.lambda1 - 12.0);
  if (!rate_ok(c->s3) || !rate_ok(c->l2)) {
    delete c;
    return CLBM_EINVAL;
  }
  c->L = L;
  c->pitch = view_pitch(p.nx, p.precision);
  c->plane = (long long)p.ny * c->pitch;
  c->buf_bytes = (size_t)planes_of(p.viscous_heating) * (size_t)c->plane * L->elem_bytes;
  c->have_walls = p.periodic_x && c->gpy;
  for (int s = 0; s < 4; ++s)
    for (int k = 0; k < 3; ++k) c->side_b[s][k] = 0.0;
  cudaError_t e;
  if (stream) {
    c->stream = static_cast<cudaStream_t>(stream);
  } else {
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete c;
      return CLBM_ECUDA;
    }
    c->own_stream = true;
  }
  if (buf_a && buf_b) {
    c->buf[0] = buf_a;
    c->buf[1] = buf_b;
    c->borrowed = true;
  }
  for (int b = 0; b < 2; ++b) {
    if (!c->borrowed) {
      e = cudaMalloc(&c->buf[b], c->buf_bytes);
      if (e != cudaSuccess) {
        cudaGetLastError();
        clbm_destroy(c);
        return e == cudaErrorMemoryAllocation ? CLBM_ENOMEM : CLBM_ECUDA;
      }
    }
    e = cudaMemsetAsync(c->buf[b], 0, c->buf_bytes, c->stream);
    if (e != cudaSuccess) {
      clbm_destroy(c);
      return CLBM_ECUDA;
    }
  }
  e = cudaMalloc(&c->d_part, sizeof(double) * (kMaxRedBlocks * 8 + 16));
  if (e != cudaSuccess) {
    cudaGetLastError();
    clbm_destroy(c);
    return CLBM_ENOMEM;
  }
  if (c->plane > (1LL << 31) - 1 || upload_boundary_list(c, {}) != cudaSuccess) {
    cudaGetLastError();
    clbm_destroy(c);
    return CLBM_ENOMEM;
  }
  clbm_status st = clbm_init_fields(c, nullptr, nullptr, nullptr, nullptr, 0);
  if (st != CLBM_OK) {
    clbm_destroy(c);
    return st;
  }
  *out = c;
  return CLBM_OK;
}

clbm_status clbm_create(const clbm_params* params, void* stream, clbm_ctx** out) {
  return create_impl(params, stream, nullptr, nullptr, out);
}

clbm_status clbm_set_boundaries(clbm_ctx* c, const uint8_t* solid, const clbm_tbc* tbc,
                                int32_t n_tbc, const int32_t* side_tbc, const clbm_link* links,
                                int32_t n_links) {
  if (!c) return CLBM_EINVAL;
  try {
    // The caller describes the whole lattice (NY rows).  A slab stores rows
    // r = 0 .. ny - 1 holding the lattice's rows y0 - 1 + r (own rows
    // [ylo, yhi), ghost rows around them); a whole lattice stores every row.
    const int nx = c->p.nx, ny = c->p.ny, NY = c->gny;
    const bool px = c->p.periodic_x, gpy = c->gpy;
    if (n_tbc < 0 || n_links < 0 || (n_tbc > 0 && !tbc) || (n_links > 0 && !links))
      return fail(c, CLBM_EINVAL, "null table with a positive count");
    for (int k = 0; k < n_tbc; ++k) {
      const clbm_tbc& b = tbc[k];
      if (!std::isfinite(b.b1) || !std::isfinite(b.b2) || !std::isfinite(b.b3) || b.b1 < 0 ||
          b.b2 < 0 || (b.b1 == 0 && b.b2 == 0))
        return fail(c, CLBM_EINVAL, "thermal condition " + std::to_string(k) +
                                        " needs b1, b2 >= 0, not both zero");
    }
    int sides[4];
    for (int s = 0; s < 4; ++s) {
      const bool periodic = s < 2 ? px : gpy;
      sides[s] = side_tbc ? side_tbc[s] : -1;
      if (!periodic && (sides[s] < 0 || sides[s] >= n_tbc))
        return fail(c, CLBM_EINVAL, "box side " + std::to_string(s) + " needs a thermal condition");
      if (periodic) sides[s] = -1;
    }
    const long long n = (long long)nx * NY;
    // lattice row of stored row r (-1: beyond a box wall, not part of the lattice)
    auto grow = [&](int r) -> int {
      if (!c->slab) return r;
      int gy = c->y0 - 1 + r;
      if (gy < 0 || gy >= NY) {
        if (!gpy) return -1;
        gy = (gy + NY) % NY;
      }
      return gy;
    };
    std::vector<uint8_t> sol;  // [ny][nx] over the stored rows
    if (solid) {
      sol.assign((size_t)ny * nx, 0);
      for (int r = 0; r < ny; ++r) {
        const int gy = grow(r);
        if (gy >= 0) std::memcpy(&sol[(size_t)r * nx], solid + (size_t)gy * nx, (size_t)nx);
      }
    }
    auto is_solid = [&](int x, int y) { return !sol.empty() && sol[(size_t)y * nx + x] != 0; };
    // listed links of own-row nodes: per node a slot with 4 directions
    std::vector<int32_t> slot_of;  // dense [ny][nx]
    std::vector<double> lk_ne;
    std::vector<int32_t> lk_tbc;
    std::vector<double> lk_q;  // 8 per slot
    std::vector<clbm_link> kept;
    const bool masked = solid != nullptr || n_links > 0;
    if (masked) slot_of.assign((size_t)ny * nx, -1);
    for (int l = 0; l < n_links; ++l) {
      const clbm_link& k = links[l];
      const bool axis = k.dir >= 1 && k.dir <= 4;
      if (k.node < 0 || k.node >= n || k.dir < 1 || k.dir > 8 || !(k.q > 0.0 && k.q <= 1.0) ||
          (axis && (k.tbc < 0 || k.tbc >= n_tbc || !(k.n_dot_e > 0) || !std::isfinite(k.n_dot_e))))
        return fail(c, CLBM_EINVAL, "bad wall link " + std::to_string(l));
      const int x = (int)(k.node % nx), gy = (int)(k.node / nx);
      if (solid && solid[k.node]) return fail(c, CLBM_EINVAL, "wall link from a solid node");
      const int y = gy - c->y0 + c->ylo;  // stored row (whole lattices: y0 = ylo = 0)
      if (y < c->ylo || y >= c->yhi) continue;  // another slab's node
      if (c->slab && axis && k.q < 0.5 && tbc[k.tbc].b1 == 0.0) {
        // the off-midpoint Dirichlet rule reads T at x_f - 2 e_i: it must be stored
        const int y3 = y + 2 * kEY[k.dir];
        const int gy3 = gy + 2 * kEY[k.dir];
        if ((y3 < 0 || y3 >= ny) && (gpy || (gy3 >= 0 && gy3 < NY)))
          return fail(c, CLBM_EINVAL, "slab too thin for wall link " + std::to_string(l) +
                                          ": its third node lies beyond the ghost row");
      }
      int32_t& s = slot_of[(size_t)y * nx + x];
      if (s < 0) {
        s = (int32_t)(lk_tbc.size() / 4);
        lk_ne.insert(lk_ne.end(), 4, 0.0);
        lk_tbc.insert(lk_tbc.end(), 4, -1);
        lk_q.insert(lk_q.end(), 8, 0.5);
      }
      if (axis) {
        lk_ne[4 * s + k.dir - 1] = k.n_dot_e;
        lk_tbc[4 * s + k.dir - 1] = k.tbc;
      }
      lk_q[8 * s + k.dir - 1] = k.q;
      clbm_link kk = k;
      kk.node = y * nx + x;
      kept.push_back(kk);
    }
    std::vector<uint16_t> flags;
    std::vector<int32_t> slot_pitch;
    if (masked) {
      flags.assign((size_t)ny * c->pitch, 0);
      slot_pitch.assign((size_t)ny * c->pitch, -1);
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          const size_t ip = (size_t)y * c->pitch + x;
          if (is_solid(x, y)) {
            flags[ip] = kFlagSolid;
            continue;
          }
          if (y < c->ylo || y >= c->yhi) continue;  // ghost rows: only their solid bits are read
          uint16_t f = 0;
          int fluid_nb = 0;
          for (int j = 1; j < 9; ++j) {
            int sx = x - kEX[j], sy = y - kEY[j];
            bool wall = false;
            if (sx < 0 || sx >= nx) {
              if (px) sx = (sx + nx) % nx; else wall = true;
            }
            if (sy < c->ylo || sy >= c->yhi) {
              if (sy < c->ylo ? c->ywlo : c->ywhi)
                wall = true;
              else if (!c->slab)
                sy = (sy + ny) % ny;  // periodic seam (slabs read their ghost row)
            }
            if (!wall && is_solid(sx, sy)) {
              wall = true;
              // a D2Q5 link into a solid needs a listed condition: link dir i = opp(j)
              if (j <= 4) {
                const int s = slot_of[(size_t)y * nx + x];
                if (s < 0 || lk_tbc[4 * s + kOpp[j] - 1] < 0)
                  return fail(c, CLBM_EINVAL, "missing wall link at node " +
                                                  std::to_string((long long)grow(y) * nx + x) +
                                                  " dir " + std::to_string(kOpp[j]));
              }
            }
            if (wall) f |= (uint16_t)(1u << (j - 1));
            else ++fluid_nb;
          }
          if (fluid_nb == 0 && n > 1)
            return fail(c, CLBM_EINVAL, "isolated fluid node " + std::to_string((long long)grow(y) * nx + x));
          const int s = slot_of[(size_t)y * nx + x];
          if (s >= 0) {
            f |= kFlagLinks;
            slot_pitch[ip] = s;
          }
          flags[ip] = f;
        }
    }
    // upload
    CLBM_CUDA(c, cudaStreamSynchronize(c->stream));
    drop_graphs(c);  // captured steps hold the old wall description
    free_tables(c);
    if (masked) {
      const size_t np = (size_t)ny * c->pitch;
      CLBM_CUDA(c, cudaMalloc(&c->d_flags, np * sizeof(uint16_t)));
      CLBM_CUDA(c, cudaMalloc(&c->d_slot, np * sizeof(int32_t)));
      CLBM_CUDA(c, cudaMemcpy(c->d_flags, flags.data(), np * sizeof(uint16_t), cudaMemcpyHostToDevice));
      CLBM_CUDA(c, cudaMemcpy(c->d_slot, slot_pitch.data(), np * sizeof(int32_t), cudaMemcpyHostToDevice));
      const size_t ns = std::max<size_t>(lk_tbc.size(), 4);
      lk_ne.resize(ns, 0.0);
      lk_tbc.resize(ns, -1);
      lk_q.resize(2 * ns, 0.5);
      CLBM_CUDA(c, cudaMalloc(&c->d_lk_ne, ns * sizeof(double)));
      CLBM_CUDA(c, cudaMalloc(&c->d_lk_tbc, ns * sizeof(int32_t)));
      CLBM_CUDA(c, cudaMalloc(&c->d_lk_q, 2 * ns * sizeof(double)));
      CLBM_CUDA(c, cudaMemcpy(c->d_lk_ne, lk_ne.data(), ns * sizeof(double), cudaMemcpyHostToDevice));
      CLBM_CUDA(c, cudaMemcpy(c->d_lk_tbc, lk_tbc.data(), ns * sizeof(int32_t), cudaMemcpyHostToDevice));
      CLBM_CUDA(c, cudaMemcpy(c->d_lk_q, lk_q.data(), 2 * ns * sizeof(double), cudaMemcpyHostToDevice));
      {  // classes of the interior kernel's warp tiles (32 vec nodes of a row): 0 = no
         // fluid node (skipped), 1 = fluid nodes only, none flagged, 2 = holds a
         // flagged node (solid, or fluid next to a wall) whose store it leaves out
        const int tw = 32 * c->L->vec;
        const int tpr = (nx + tw - 1) / tw;
        std::vector<uint8_t> tf((size_t)ny * tpr, 0), flagged((size_t)ny * tpr, 0);
        for (int y = 0; y < ny; ++y)
          for (int x = 0; x < nx; ++x) {
            const uint16_t f = flags[(size_t)y * c->pitch + x];
            const size_t t = (size_t)y * tpr + x / tw;
            if (!(f & kFlagSolid)) tf[t] = 1;
            if (f) flagged[t] = 1;
          }
        for (size_t t = 0; t < tf.size(); ++t)
          if (tf[t] && flagged[t]) tf[t] = 2;
        CLBM_CUDA(c, cudaMalloc(&c->d_tile_fluid, tf.size()));
        CLBM_CUDA(c, cudaMemcpy(c->d_tile_fluid, tf.data(), tf.size(), cudaMemcpyHostToDevice));
        c->tiles_per_row = tpr;
      }
    }
    {
      std::vector<double> t3((size_t)std::max(n_tbc, 1) * 3, 0.0);
      for (int k = 0; k < n_tbc; ++k) {
        t3[3 * k] = tbc[k].b1;
        t3[3 * k + 1] = tbc[k].b2;
        t3[3 * k + 2] = tbc[k].b3;
      }
      CLBM_CUDA(c, cudaMalloc(&c->d_tbc, t3.size() * sizeof(double)));
      CLBM_CUDA(c, cudaMemcpy(c->d_tbc, t3.data(), t3.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    CLBM_CUDA(c, upload_boundary_list(c, flags));
    for (int s = 0; s < 4; ++s) {
      c->side_tbc[s] = sides[s];
      for (int k = 0; k < 3; ++k)
        c->side_b[s][k] = sides[s] >= 0 ? (&tbc[sides[s]].b1)[k] : 0.0;
    }
    c->h_solid = std::move(sol);
    c->h_tbc.assign(tbc, tbc + n_tbc);
    c->h_links = std::move(kept);
    c->have_walls = true;
    return CLBM_OK;
  } catch (const std::bad_alloc&) {
    return fail(c, CLBM_ENOMEM, "host allocation failed");
  } catch (...) {
    return fail(c, CLBM_EINVAL, "unexpected host error");
  }
}

static clbm_status ensure_fields_scratch(clbm_ctx* c) {
  if (c->d_fields) return CLBM_OK;
  const size_t n = (size_t)c->p.nx * (c->yhi - c->ylo);
  cudaError_t e = cudaMalloc(&c->d_fields, 4 * n * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->d_fields = nullptr;
    return fail(c, CLBM_ENOMEM, "cannot allocate the field scratch");
  }
  return CLBM_OK;
}

// The device's view of a host buffer that kernels may read and write in place:
// page-locked host memory mapped into the device's address space (on a
// Grace-Blackwell node the GPU reaches it coherently over NVLink-C2C, at the
// rate of the copy engines).  nullptr for pageable memory.
static void* mapped_view(const void* p) {
  cudaPointerAttributes a;
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

clbm_status clbm_init_fields(clbm_ctx* c, const double* rho, const double* ux, const double* uy,
                             const double* T, int32_t on_device) {
  if (!c) return CLBM_EINVAL;
  const size_t n = (size_t)c->p.nx * (c->yhi - c->ylo);
  const double* src[4] = {rho, ux, uy, T};
  const double* dev[4] = {nullptr, nullptr, nullptr, nullptr};
  if (on_device) {
    for (int k = 0; k < 4; ++k) dev[k] = src[k];
  } else if (rho || ux || uy || T) {
    // mapped page-locked fields are read by the kernel itself, so the
    // transfer overlaps the initialisation; pageable ones go through the scratch
    for (int k = 0; k < 4; ++k) {
      if (!src[k]) continue;
      dev[k] = static_cast<const double*>(mapped_view(src[k]));
      if (dev[k]) continue;
      clbm_status st = ensure_fields_scratch(c);
      if (st != CLBM_OK) return st;
      double* d = c->d_fields + k * n;
      CLBM_CUDA(c, cudaMemcpyAsync(d, src[k], n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
      dev[k] = d;
    }
  }
  CLBM_CUDA(c, c->L->init(make_geom(c), make_coef(c), c->buf[0], dev[0], dev[1], dev[2], dev[3],
                          c->stream));
  c->cur = 0;
  c->t = 0;
  if (!on_device && (rho || ux || uy || T)) CLBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return CLBM_OK;
}

static StepArgs step_args(const clbm_ctx* c, int cur, int64_t t) {
  StepArgs a;
  a.g = make_geom(c);
  a.c = make_coef(c);
  a.stochastic = c->p.rounding;
  a.bnodes = c->d_bnodes;
  a.nb = (int)c->h_bnodes.size();
  a.src = c->buf[cur];
  a.dst = c->buf[cur ^ 1];
  a.seed = (uint32_t)(t * 0x9E3779B1ull) ^ (uint32_t)(t >> 32);
  a.reverse = (int)(t & 1);
  a.tdev = nullptr;
  a.tstep = 0;
  return a;
}

// Capture `len` steps starting from buffer `cur` at a step of parity `par`.
static clbm_status capture_steps(clbm_ctx* c, int cur, int par, int len, cudaGraphExec_t* out) {
  if (!c->d_t) CLBM_CUDA(c, cudaMalloc(&c->d_t, sizeof(long long)));
  cudaGraph_t graph;
  CLBM_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int j = 0; j < len && e == cudaSuccess; ++j) {
    StepArgs a = step_args(c, (cur + j) & 1, par + j);
    a.tdev = c->d_t;
    a.tstep = j;
    e = c->L->step(a, c->stream);
  }
  if (e == cudaSuccess) e = launch_advance(c->d_t, len, c->stream);
  cudaError_t e2 = cudaStreamEndCapture(c->stream, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (e2 == cudaSuccess) cudaGraphDestroy(graph);
    cudaGetLastError();
    return cuda_fail(c, e != cudaSuccess ? e : e2, "capture of the step graph");
  }
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(c, e, "instantiate the step graph");
  return CLBM_OK;
}

clbm_status clbm_step(clbm_ctx* c, int64_t nsteps) {
  if (!c || nsteps < 0) return fail(c, CLBM_EINVAL, "bad step count");
  if (!c->have_walls) return fail(c, CLBM_EINVAL, "non-periodic lattice: call clbm_set_boundaries first");
  // Runs of two or more steps replay captured graphs of 32, 16, ..., 2 steps
  // (the binary digits of nsteps; fewer launch gaps), with the step count on
  // the device.  Every graph length is even, so the buffer/parity key stays the
  // same across them; the graphs of a key and of the key one single step away
  // are captured together on first use, so later calls of any length start
  // without a capture.  Not while the caller is capturing the stream itself.
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CLBM_CUDA(c, cudaStreamIsCapturing(c->stream, &cs));
  if (nsteps >= 2 && cs == cudaStreamCaptureStatusNone) {
    const int key = c->cur * 2 + (int)(c->t & 1);
    for (const int k : {key, key ^ 3})
      for (int l = 0; l < kGraphLevels; ++l)
        if (!c->step_graph[k][l]) {
          clbm_status st = capture_steps(c, k >> 1, k & 1, 2 << l, &c->step_graph[k][l]);
          if (st != CLBM_OK) return st;
        }
    CLBM_CUDA(c, launch_set_step(c->d_t, c->t, c->stream));
    while (nsteps >= kGraphSteps) {
      CLBM_CUDA(c, cudaGraphLaunch(c->step_graph[key][kGraphLevels - 1], c->stream));
      c->t += kGraphSteps;  // even: the current buffer is unchanged
      nsteps -= kGraphSteps;
    }
    for (int l = kGraphLevels - 2; l >= 0; --l)
      if (nsteps >= (2 << l)) {
        CLBM_CUDA(c, cudaGraphLaunch(c->step_graph[key][l], c->stream));
        c->t += 2 << l;
        nsteps -= 2 << l;
      }
  }
  for (int64_t s = 0; s < nsteps; ++s) {
    StepArgs a = step_args(c, c->cur, c->t);
    cudaError_t e = c->L->step(a, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "step kernel launch");
    c->cur ^= 1;
    c->t += 1;
  }
  return CLBM_OK;
}

clbm_status clbm_create_slab(const clbm_params* params, int32_t y0, int32_t rows, void* stream,
                             clbm_ctx** out) {
  SlabSpec sp{y0, rows};
  return create_impl(params, stream, nullptr, nullptr, out, &sp);
}

static int plane_count(const clbm_ctx* c) { return planes_of(c->p.viscous_heating); }

clbm_status clbm_halo_bytes(const clbm_ctx* c, int64_t* bytes) {
  if (!c || !bytes) return CLBM_EINVAL;
  *bytes = (int64_t)plane_count(c) * c->p.nx * (int64_t)c->L->elem_bytes;
  return CLBM_OK;
}

// One row of every plane of the current state.
static char* row_ptr(const clbm_ctx* c, int row) {
  return static_cast<char*>(c->buf[c->cur]) + (size_t)row * c->pitch * c->L->elem_bytes;
}

clbm_status clbm_halo_pack(clbm_ctx* c, int32_t side, void* dst) {
  if (!c || !dst || (side != 0 && side != 1) || !c->slab) return fail(c, CLBM_EINVAL, "bad halo pack");
  const size_t eb = c->L->elem_bytes, w = (size_t)c->p.nx * eb;
  CLBM_CUDA(c, cudaMemcpy2DAsync(dst, w, row_ptr(c, side ? c->yhi - 1 : c->ylo), c->plane * eb, w,
                                 plane_count(c), cudaMemcpyDeviceToDevice, c->stream));
  return CLBM_OK;
}

clbm_status clbm_halo_unpack(clbm_ctx* c, int32_t side, const void* src) {
  if (!c || !src || (side != 0 && side != 1) || !c->slab) return fail(c, CLBM_EINVAL, "bad halo unpack");
  const size_t eb = c->L->elem_bytes, w = (size_t)c->p.nx * eb;
  CLBM_CUDA(c, cudaMemcpy2DAsync(row_ptr(c, side ? c->yhi : c->ylo - 1), c->plane * eb, src, w, w,
                                 plane_count(c), cudaMemcpyDeviceToDevice, c->stream));
  return CLBM_OK;
}

clbm_status clbm_halo_copy(clbm_ctx* from, int32_t side, clbm_ctx* to) {
  if (!from || !to || (side != 0 && side != 1) || !from->slab || !to->slab)
    return fail(to, CLBM_EINVAL, "bad halo copy");
  if (from->p.nx != to->p.nx || from->L != to->L || plane_count(from) != plane_count(to))
    return fail(to, CLBM_EINVAL, "halo copy between different lattices");
  const size_t eb = from->L->elem_bytes, w = (size_t)from->p.nx * eb;
  const bool two = from->stream != to->stream;
  if (two) {  // the copy waits for `from`'s step; `from`'s next writes wait for the copy
    for (clbm_ctx* k : {from, to})
      if (!k->ev_halo[0]) {
        CLBM_CUDA(to, cudaEventCreateWithFlags(&k->ev_halo[0], cudaEventDisableTiming));
        CLBM_CUDA(to, cudaEventCreateWithFlags(&k->ev_halo[1], cudaEventDisableTiming));
      }
    CLBM_CUDA(to, cudaEventRecord(from->ev_halo[0], from->stream));
    CLBM_CUDA(to, cudaStreamWaitEvent(to->stream, from->ev_halo[0], 0));
  }
  // side 0: `from`'s first own row -> the ghost row above `to` (the slab below);
  // side 1: its last own row -> the ghost row below `to` (the slab above)
  CLBM_CUDA(to, cudaMemcpy2DAsync(row_ptr(to, side ? to->ylo - 1 : to->yhi), to->plane * eb,
                                  row_ptr(from, side ? from->yhi - 1 : from->ylo), from->plane * eb, w,
                                  plane_count(from), cudaMemcpyDefault, to->stream));
  if (two) {
    CLBM_CUDA(to, cudaEventRecord(to->ev_halo[1], to->stream));
    CLBM_CUDA(to, cudaStreamWaitEvent(from->stream, to->ev_halo[1], 0));
  }
  return CLBM_OK;
}

clbm_status clbm_slabs_exchange(clbm_ctx* const* slabs, int32_t n, int32_t periodic) {
  if (!slabs || n < 1) return CLBM_EINVAL;
  for (int k = 0; k < n; ++k)
    if (!slabs[k] || !slabs[k]->slab) return CLBM_EINVAL;
  // One stream, one device, one format: every seam in one kernel launch (the
  // rows are copied whole, pitch included, so the copies are 16-byte words).
  bool one = 2 * n <= kMaxHaloCopies;
  for (int k = 1; k < n && one; ++k)
    one = slabs[k]->stream == slabs[0]->stream && slabs[k]->L == slabs[0]->L &&
          slabs[k]->pitch == slabs[0]->pitch && plane_count(slabs[k]) == plane_count(slabs[0]);
  if (one) {
    HaloTable t{};
    const size_t eb = slabs[0]->L->elem_bytes;
    t.planes = plane_count(slabs[0]);
    t.row_bytes = (long long)slabs[0]->pitch * (long long)eb;
    for (int k = 0; k < n; ++k) {
      const int up = k + 1 < n ? k + 1 : (periodic ? 0 : -1);
      if (up < 0) continue;
      clbm_ctx *a = slabs[k], *b = slabs[up];
      // a's last own row -> the ghost row below b; b's first own row -> the ghost row above a
      t.c[t.n++] = HaloCopy{row_ptr(a, a->yhi - 1), row_ptr(b, b->ylo - 1), a->plane * (long long)eb,
                            b->plane * (long long)eb};
      t.c[t.n++] = HaloCopy{row_ptr(b, b->ylo), row_ptr(a, a->yhi), b->plane * (long long)eb,
                            a->plane * (long long)eb};
    }
    CLBM_CUDA(slabs[0], launch_halo(t, slabs[0]->stream));
    return CLBM_OK;
  }
  for (int k = 0; k < n; ++k) {
    const int up = k + 1 < n ? k + 1 : (periodic ? 0 : -1);
    if (up < 0) continue;
    clbm_status st = clbm_halo_copy(slabs[k], 1, slabs[up]);  // k's top row below `up`
    if (st != CLBM_OK) return st;
    st = clbm_halo_copy(slabs[up], 0, slabs[k]);  // `up`'s bottom row above k
    if (st != CLBM_OK) return st;
  }
  return CLBM_OK;
}

clbm_status clbm_slabs_step(clbm_ctx* const* slabs, int32_t n, int32_t periodic, int64_t nsteps) {
  if (!slabs || n < 1 || nsteps < 0) return CLBM_EINVAL;
  for (int64_t s = 0; s < nsteps; ++s) {
    for (int k = 0; k < n; ++k) {
      clbm_status st = clbm_step(slabs[k], 1);
      if (st != CLBM_OK) return st;
    }
    clbm_status st = clbm_slabs_exchange(slabs, n, periodic);
    if (st != CLBM_OK) return st;
  }
  return CLBM_OK;
}

clbm_status clbm_set_wall_velocity(clbm_ctx* c, int32_t side, double ux, double uy) {
  if (!c || side < 0 || side > 3 || !std::isfinite(ux) || !std::isfinite(uy))
    return fail(c, CLBM_EINVAL, "bad wall velocity");
  CLBM_CUDA(c, cudaStreamSynchronize(c->stream));
  drop_graphs(c);  // captured steps hold the old wall description
  c->side_u[side][0] = ux;
  c->side_u[side][1] = uy;
  return CLBM_OK;
}

clbm_status clbm_damp_period2(clbm_ctx* c) {
  if (!c) return CLBM_EINVAL;
  if (c->t < 1) return fail(c, CLBM_EINVAL, "needs one step after initialisation");
  CLBM_CUDA(c, c->L->average(c->buf[c->cur], c->buf[c->cur ^ 1],
                             planes_of(c->p.viscous_heating) * c->plane, c->stream));
  return CLBM_OK;
}

clbm_status clbm_time(const clbm_ctx* c, int64_t* t_out) {
  if (!c || !t_out) return CLBM_EINVAL;
  *t_out = c->t;
  return CLBM_OK;
}

clbm_status clbm_field_shape(const clbm_ctx* c, int64_t* nx_out, int64_t* rows_out) {
  if (!c || !nx_out || !rows_out) return CLBM_EINVAL;
  *nx_out = c->p.nx;
  *rows_out = c->yhi - c->ylo;
  return CLBM_OK;
}

clbm_status clbm_moments(clbm_ctx* c, double* rho, double* ux, double* uy, double* T,
                         int32_t on_device) {
  if (!c) return CLBM_EINVAL;
  const size_t n = (size_t)c->p.nx * (c->yhi - c->ylo);
  if (on_device) {
    CLBM_CUDA(c, c->L->moments(make_geom(c), make_coef(c), c->buf[c->cur], rho, ux, uy, T, c->stream));
    return CLBM_OK;
  }
  // the kernel writes mapped page-locked outputs in place; pageable ones are
  // written to the scratch and copied
  double* d[4];
  bool staged[4] = {false, false, false, false};
  double* h[4] = {rho, ux, uy, T};
  for (int k = 0; k < 4; ++k) {
    d[k] = h[k] ? static_cast<double*>(mapped_view(h[k])) : nullptr;
    if (!h[k] || d[k]) continue;
    clbm_status st = ensure_fields_scratch(c);
    if (st != CLBM_OK) return st;
    d[k] = c->d_fields + k * n;
    staged[k] = true;
  }
  CLBM_CUDA(c, c->L->moments(make_geom(c), make_coef(c), c->buf[c->cur], d[0], d[1], d[2], d[3],
                             c->stream));
  for (int k = 0; k < 4; ++k)
    if (staged[k]) CLBM_CUDA(c, cudaMemcpyAsync(h[k], d[k], n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CLBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return CLBM_OK;
}

static int red_blocks(long long work) {
  long long b = (work + 255) / 256;
  return (int)std::max(1LL, std::min<long long>(b, kMaxRedBlocks));
}

// The Nusselt link list of a selection (built on the host once, then cached):
// which = 0..3 a box side, 4 + k the listed links with condition k.  A slab
// lists only its own nodes' links (none for a box side it does not touch).
static clbm_status nusselt_list(clbm_ctx* c, int which, const NuLink** out, int* count) {
  auto it = c->nu_lists.find(which);
  if (it == c->nu_lists.end()) {
    const int nx = c->p.nx, pitch = c->pitch;
    const bool px = c->p.periodic_x;
    auto solid = [&](int x, int y) { return !c->h_solid.empty() && c->h_solid[(size_t)y * nx + x]; };
    auto second = [&](int x, int y, int dx, int dy) -> long long {
      int x2 = x + dx, y2 = y + dy;
      if (x2 < 0 || x2 >= nx) {
        if (!px) return -1;
        x2 = (x2 + nx) % nx;
      }
      if (y2 < c->ylo || y2 >= c->yhi) {
        if (y2 < c->ylo ? c->ywlo : c->ywhi) return -1;  // beyond a box wall
        if (!c->slab) y2 = (y2 + c->p.ny) % c->p.ny;     // periodic seam (slabs: ghost row)
      }
      if (solid(x2, y2)) return -1;
      return (long long)y2 * pitch + x2;
    };
    std::vector<NuLink> v;
    if (which < 4) {
      if (c->side_tbc[which] < 0) return fail(c, CLBM_EINVAL, "periodic side has no wall");
      const clbm_tbc& b = c->h_tbc[c->side_tbc[which]];
      // link direction i toward the wall: x0 -> 3, x1 -> 1, y0 -> 4, y1 -> 2
      const int i = which == 0 ? 3 : which == 1 ? 1 : which == 2 ? 4 : 2;
      const bool here = which < 2 || (which == 2 ? c->ywlo : c->ywhi);
      const int cnt = !here ? 0 : (which < 2 ? c->yhi - c->ylo : nx);
      for (int k = 0; k < cnt; ++k) {
        const int x = which == 0 ? 0 : which == 1 ? nx - 1 : k;
        const int y = which == 2 ? c->ylo : which == 3 ? c->yhi - 1 : c->ylo + k;
        if (solid(x, y)) continue;
        NuLink L;
        L.own = (long long)y * pitch + x;
        L.second = second(x, y, -kEX[i], -kEY[i]);
        L.ne = 1.0;
        L.b1 = b.b1;
        L.b2 = b.b2;
        L.b3 = b.b3;
        L.q = 0.5;
        v.push_back(L);
      }
    } else {
      const int t = which - 4;
      if (t >= (int)c->h_tbc.size()) return fail(c, CLBM_EINVAL, "no such thermal condition");
      for (const clbm_link& k : c->h_links) {
        if (k.dir > 4 || k.tbc != t) continue;  // diagonal links carry only q
        const int x = (int)(k.node % nx), y = (int)(k.node / nx);
        const clbm_tbc& b = c->h_tbc[t];
        NuLink L;
        L.own = (long long)y * pitch + x;
        L.second = second(x, y, -kEX[k.dir], -kEY[k.dir]);
        L.ne = k.n_dot_e;
        L.b1 = b.b1;
        L.b2 = b.b2;
        L.b3 = b.b3;
        L.q = k.q;
        v.push_back(L);
      }
    }
    NuLink* d = nullptr;
    if (!v.empty()) {
      CLBM_CUDA(c, cudaMalloc(&d, v.size() * sizeof(NuLink)));
      cudaError_t e = cudaMemcpy(d, v.data(), v.size() * sizeof(NuLink), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(c, e, "upload Nusselt links");
      }
    }
    it = c->nu_lists.emplace(which, std::make_pair(d, (int)v.size())).first;
  }
  *out = it->second.first;
  *count = it->second.second;
  return CLBM_OK;
}

// Raw FP64 sums of one reduction over the own rows (the residual, Nusselt and
// conservation entry points finish these; slabs of one lattice add theirs first).
static clbm_status reduce_sums(clbm_ctx* c, int what, int which, double* out) {
  double* red = c->d_part + kMaxRedBlocks * 8;
  int width = 8;
  if (what == 0) {  // residual: dT^2, T^2, dux^2, ux^2, duy^2, uy^2, non-finite count
    if (c->t < 1) return fail(c, CLBM_EINVAL, "residual needs one step after initialisation");
    const int nb = red_blocks((long long)c->p.nx * (c->yhi - c->ylo));
    CLBM_CUDA(c, c->L->residual(make_geom(c), make_coef(c), c->buf[c->cur], c->buf[c->cur ^ 1],
                                c->d_part, nb, c->stream));
    CLBM_CUDA(c, launch_reduce_partials(c->d_part, nb, 8, red, c->stream));
  } else if (what == 1) {  // Nusselt: sum of dT/dn, link count, non-finite count
    if (!c->have_walls) return fail(c, CLBM_EINVAL, "no walls");
    const NuLink* links = nullptr;
    int nl = 0;
    clbm_status st = nusselt_list(c, which, &links, &nl);
    if (st != CLBM_OK) return st;
    for (int k = 0; k < 8; ++k) out[k] = 0.0;
    if (nl == 0) return CLBM_OK;
    const int nb = red_blocks(nl);
    CLBM_CUDA(c, c->L->nusselt(make_geom(c), make_coef(c), c->buf[c->cur], links, nl, c->d_part, nb,
                               c->stream));
    CLBM_CUDA(c, launch_reduce_partials(c->d_part, nb, 2, red, c->stream));
    double h[2];
    CLBM_CUDA(c, cudaMemcpyAsync(h, red, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    CLBM_CUDA(c, cudaStreamSynchronize(c->stream));
    out[0] = h[0];
    out[1] = (double)nl;
    out[2] = h[1];
    return CLBM_OK;
  } else if (what == 2) {  // totals: sum d_i, d_i e_ix, d_i e_iy, h_j, fluid count, non-finite count
    const int nb = red_blocks((long long)c->p.nx * (c->yhi - c->ylo));
    CLBM_CUDA(c, c->L->totals(make_geom(c), c->buf[c->cur], c->d_part, nb, c->stream));
    CLBM_CUDA(c, launch_reduce_partials(c->d_part, nb, 8, red, c->stream));
  } else {
    return fail(c, CLBM_EINVAL, "unknown reduction");
  }
  CLBM_CUDA(c, cudaMemcpyAsync(out, red, width * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CLBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return CLBM_OK;
}

static clbm_status finish_sums(const clbm_ctx* c, int what, const double* h, double length,
                               double dT, double* out) {
  if (what == 0) {
    if (h[6] != 0.0 || !std::isfinite(h[0] + h[1] + h[2] + h[3] + h[4] + h[5])) {
      out[0] = INFINITY;
      return CLBM_EUNSTABLE;
    }
    double best = 0.0;
    for (int k = 0; k < 3; ++k) {
      const double v = std::sqrt(h[2 * k]) / std::max(std::sqrt(h[2 * k + 1]), 1e-30);
      best = std::max(best, v);
    }
    out[0] = best;
    return CLBM_OK;
  }
  if (what == 1) {
    if (!(h[1] > 0)) return CLBM_EINVAL;
    if (h[2] != 0.0) {
      out[0] = NAN;
      return CLBM_EUNSTABLE;
    }
    out[0] = length / dT * (h[0] / h[1]);
    return CLBM_OK;
  }
  if (what == 2) {
    // the stored values are deviations from the rest state: f_i = w_i rho0 + d_i,
    // g_j = w_j T0 + h_j (the rest state carries no momentum)
    out[0] = h[4] * c->p.rho0 + h[0];
    out[1] = h[1];
    out[2] = h[2];
    out[3] = h[4] * c->p.T0 + h[3];
    if (h[5] != 0.0 || !std::isfinite(out[0] + out[1] + out[2] + out[3])) return CLBM_EUNSTABLE;
    return CLBM_OK;
  }
  return CLBM_EINVAL;
}

clbm_status clbm_reduce_sums(clbm_ctx* c, int32_t what, int32_t which, double* out) {
  if (!c || !out) return fail(c, CLBM_EINVAL, "bad reduction arguments");
  try {
    return reduce_sums(c, what, which, out);
  } catch (const std::bad_alloc&) {
    return fail(c, CLBM_ENOMEM, "host allocation failed");
  }
}

clbm_status clbm_finish_sums(const clbm_ctx* c, int32_t what, const double* sums, double length,
                             double dT, double* out) {
  if (!c || !sums || !out || (what == 1 && !(dT != 0)) || !std::isfinite(length)) return CLBM_EINVAL;
  return finish_sums(c, what, sums, length, dT, out);
}

clbm_status clbm_nusselt(clbm_ctx* c, int32_t which, double length, double dT, double* nu_out) {
  if (!c || !nu_out || which < 0 || !(dT != 0) || !std::isfinite(length))
    return fail(c, CLBM_EINVAL, "bad Nusselt arguments");
  double h[8];
  clbm_status st = clbm_reduce_sums(c, 1, which, h);
  if (st != CLBM_OK) return st;
  if (!(h[1] > 0)) return fail(c, CLBM_EINVAL, "selection has no wall links");
  st = finish_sums(c, 1, h, length, dT, nu_out);
  if (st == CLBM_EUNSTABLE) return fail(c, st, "non-finite wall gradient");
  return st;
}

clbm_status clbm_residual(clbm_ctx* c, double* r_out) {
  if (!c || !r_out) return fail(c, CLBM_EINVAL, "bad residual arguments");
  double h[8];
  clbm_status st = clbm_reduce_sums(c, 0, 0, h);
  if (st != CLBM_OK) return st;
  st = finish_sums(c, 0, h, 0.0, 1.0, r_out);
  if (st == CLBM_EUNSTABLE) return fail(c, st, "non-finite field values");
  return st;
}

clbm_status clbm_totals(clbm_ctx* c, double* out) {
  if (!c || !out) return fail(c, CLBM_EINVAL, "bad totals arguments");
  double h[8];
  clbm_status st = clbm_reduce_sums(c, 2, 0, h);
  if (st != CLBM_OK) return st;
  st = finish_sums(c, 2, h, 0.0, 1.0, out);
  if (st == CLBM_EUNSTABLE) return fail(c, st, "non-finite field values");
  return st;
}

}  // extern "C"

namespace clbm {

int view_pitch(int nx, int precision) {
  const Launchers* L = launchers_for(precision);
  const int gran = 32 * (L ? L->vec : 4);
  return (nx + gran - 1) / gran * gran;
}

size_t view_buffer_bytes(int nx, int ny, int precision, int vh) {
  const Launchers* L = launchers_for(precision);
  if (!L) return 0;
  return (size_t)planes_of(vh) * (size_t)ny * (size_t)view_pitch(nx, precision) * L->elem_bytes;
}

clbm_status create_view(const clbm_params* p, cudaStream_t s, void* buf_a, void* buf_b,
                        clbm_ctx** out) {
  if (!buf_a || !buf_b || !s) return CLBM_EINVAL;
  return create_impl(p, s, buf_a, buf_b, out);
}

ViewInfo describe_view(const clbm_ctx* c) {
  ViewInfo v;
  v.g = make_geom(c);
  v.c = make_coef(c);
  v.buf[0] = c->buf[0];
  v.buf[1] = c->buf[1];
  v.pitch = c->pitch;
  v.plane = c->plane;
  v.bnodes_host = c->h_bnodes.data();
  v.nb = (int)c->h_bnodes.size();
  return v;
}

void set_view_time(clbm_ctx* c, int64_t t, int cur) {
  c->t = t;
  c->cur = cur;
}

}  // namespace clbm
