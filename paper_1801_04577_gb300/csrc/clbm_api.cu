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
  std::vector<uint8_t> h_solid;
  std::vector<clbm_tbc> h_tbc;
  std::vector<clbm_link> h_links;
  int side_tbc[4] = {-1, -1, -1, -1};
  double side_b[4][3] = {};
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
  const int nx = c->p.nx, ny = c->p.ny;
  const bool py = c->p.periodic_y;
  std::vector<int32_t>& v = c->h_bnodes;
  v.clear();
  for (int y = 0; y < ny; ++y) {
    const bool yedge = !py && (y == 0 || y == ny - 1);
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
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
  return CLBM_OK;
}

static clbm_status create_impl(const clbm_params* params, void* stream, void* buf_a, void* buf_b,
                               clbm_ctx** out) {
  if (!out) return CLBM_EINVAL;
  *out = nullptr;
  if (!params) return CLBM_EINVAL;
  const clbm_params& p = *params;
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
  c->have_walls = p.periodic_x && p.periodic_y;
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
    const int nx = c->p.nx, ny = c->p.ny;
    const bool px = c->p.periodic_x, py = c->p.periodic_y;
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
      const bool periodic = s < 2 ? px : py;
      sides[s] = side_tbc ? side_tbc[s] : -1;
      if (!periodic && (sides[s] < 0 || sides[s] >= n_tbc))
        return fail(c, CLBM_EINVAL, "box side " + std::to_string(s) + " needs a thermal condition");
      if (periodic) sides[s] = -1;
    }
    const long long n = (long long)nx * ny;
    std::vector<uint8_t> sol;
    if (solid) sol.assign(solid, solid + n);
    auto is_solid = [&](int x, int y) { return !sol.empty() && sol[(size_t)y * nx + x] != 0; };
    // listed links: per node a slot with 4 directions
    std::vector<int32_t> slot_of;  // dense [ny][nx]
    std::vector<double> lk_ne;
    std::vector<int32_t> lk_tbc;
    std::vector<double> lk_q;  // 8 per slot
    const bool masked = !sol.empty() || n_links > 0;
    if (masked) slot_of.assign((size_t)n, -1);
    for (int l = 0; l < n_links; ++l) {
      const clbm_link& k = links[l];
      const bool axis = k.dir >= 1 && k.dir <= 4;
      if (k.node < 0 || k.node >= n || k.dir < 1 || k.dir > 8 || !(k.q > 0.0 && k.q <= 1.0) ||
          (axis && (k.tbc < 0 || k.tbc >= n_tbc || !(k.n_dot_e > 0) || !std::isfinite(k.n_dot_e))))
        return fail(c, CLBM_EINVAL, "bad wall link " + std::to_string(l));
      const int x = (int)(k.node % nx), y = (int)(k.node / nx);
      if (is_solid(x, y)) return fail(c, CLBM_EINVAL, "wall link from a solid node");
      int32_t& s = slot_of[(size_t)k.node];
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
          uint16_t f = 0;
          int fluid_nb = 0;
          for (int j = 1; j < 9; ++j) {
            int sx = x - kEX[j], sy = y - kEY[j];
            bool wall = false;
            if (sx < 0 || sx >= nx) {
              if (px) sx = (sx + nx) % nx; else wall = true;
            }
            if (sy < 0 || sy >= ny) {
              if (py) sy = (sy + ny) % ny; else wall = true;
            }
            if (!wall && is_solid(sx, sy)) {
              wall = true;
              // a D2Q5 link into a solid needs a listed condition: link dir i = opp(j)
              if (j <= 4) {
                const int s = slot_of[(size_t)y * nx + x];
                if (s < 0 || lk_tbc[4 * s + kOpp[j] - 1] < 0)
                  return fail(c, CLBM_EINVAL, "missing wall link at node " +
                                                  std::to_string((long long)y * nx + x) +
                                                  " dir " + std::to_string(kOpp[j]));
              }
            }
            if (wall) f |= (uint16_t)(1u << (j - 1));
            else ++fluid_nb;
          }
          if (fluid_nb == 0 && n > 1)
            return fail(c, CLBM_EINVAL, "isolated fluid node " + std::to_string((long long)y * nx + x));
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
    c->h_links.assign(links, links + n_links);
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
  const size_t n = (size_t)c->p.nx * c->p.ny;
  cudaError_t e = cudaMalloc(&c->d_fields, 4 * n * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->d_fields = nullptr;
    return fail(c, CLBM_ENOMEM, "cannot allocate the field scratch");
  }
  return CLBM_OK;
}

clbm_status clbm_init_fields(clbm_ctx* c, const double* rho, const double* ux, const double* uy,
                             const double* T, int32_t on_device) {
  if (!c) return CLBM_EINVAL;
  const size_t n = (size_t)c->p.nx * c->p.ny;
  const double* src[4] = {rho, ux, uy, T};
  const double* dev[4] = {nullptr, nullptr, nullptr, nullptr};
  if (on_device) {
    for (int k = 0; k < 4; ++k) dev[k] = src[k];
  } else if (rho || ux || uy || T) {
    clbm_status st = ensure_fields_scratch(c);
    if (st != CLBM_OK) return st;
    for (int k = 0; k < 4; ++k) {
      if (!src[k]) continue;
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

clbm_status clbm_moments(clbm_ctx* c, double* rho, double* ux, double* uy, double* T,
                         int32_t on_device) {
  if (!c) return CLBM_EINVAL;
  const size_t n = (size_t)c->p.nx * c->p.ny;
  if (on_device) {
    CLBM_CUDA(c, c->L->moments(make_geom(c), make_coef(c), c->buf[c->cur], rho, ux, uy, T, c->stream));
    return CLBM_OK;
  }
  clbm_status st = ensure_fields_scratch(c);
  if (st != CLBM_OK) return st;
  double* d[4];
  double* h[4] = {rho, ux, uy, T};
  for (int k = 0; k < 4; ++k) d[k] = h[k] ? c->d_fields + k * n : nullptr;
  CLBM_CUDA(c, c->L->moments(make_geom(c), make_coef(c), c->buf[c->cur], d[0], d[1], d[2], d[3],
                             c->stream));
  for (int k = 0; k < 4; ++k)
    if (h[k]) CLBM_CUDA(c, cudaMemcpyAsync(h[k], d[k], n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CLBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return CLBM_OK;
}

static int red_blocks(long long work) {
  long long b = (work + 255) / 256;
  return (int)std::max(1LL, std::min<long long>(b, kMaxRedBlocks));
}

clbm_status clbm_nusselt(clbm_ctx* c, int32_t which, double length, double dT, double* nu_out) {
  if (!c || !nu_out || which < 0 || !(dT != 0) || !std::isfinite(length))
    return fail(c, CLBM_EINVAL, "bad Nusselt arguments");
  if (!c->have_walls) return fail(c, CLBM_EINVAL, "no walls");
  try {
    auto it = c->nu_lists.find(which);
    if (it == c->nu_lists.end()) {
      const int nx = c->p.nx, ny = c->p.ny, pitch = c->pitch;
      const bool px = c->p.periodic_x, py = c->p.periodic_y;
      auto solid = [&](int x, int y) { return !c->h_solid.empty() && c->h_solid[(size_t)y * nx + x]; };
      auto second = [&](int x, int y, int dx, int dy) -> long long {
        int x2 = x + dx, y2 = y + dy;
        if (x2 < 0 || x2 >= nx) {
          if (!px) return -1;
          x2 = (x2 + nx) % nx;
        }
        if (y2 < 0 || y2 >= ny) {
          if (!py) return -1;
          y2 = (y2 + ny) % ny;
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
        const int cnt = which < 2 ? ny : nx;
        for (int k = 0; k < cnt; ++k) {
          const int x = which == 0 ? 0 : which == 1 ? nx - 1 : k;
          const int y = which == 2 ? 0 : which == 3 ? ny - 1 : (which < 2 ? k : 0);
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
      if (v.empty()) return fail(c, CLBM_EINVAL, "selection has no wall links");
      NuLink* d = nullptr;
      CLBM_CUDA(c, cudaMalloc(&d, v.size() * sizeof(NuLink)));
      cudaError_t e = cudaMemcpy(d, v.data(), v.size() * sizeof(NuLink), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(c, e, "upload Nusselt links");
      }
      it = c->nu_lists.emplace(which, std::make_pair(d, (int)v.size())).first;
    }
    const int nl = it->second.second;
    const int nb = red_blocks(nl);
    double* out = c->d_part + kMaxRedBlocks * 8;
    CLBM_CUDA(c, c->L->nusselt(make_geom(c), make_coef(c), c->buf[c->cur], it->second.first, nl,
                               c->d_part, nb, c->stream));
    CLBM_CUDA(c, launch_reduce_partials(c->d_part, nb, 2, out, c->stream));
    double h[2];
    CLBM_CUDA(c, cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    CLBM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (h[1] != 0.0) {
      *nu_out = NAN;
      return fail(c, CLBM_EUNSTABLE, "non-finite wall gradient");
    }
    *nu_out = length / dT * (h[0] / (double)nl);
    return CLBM_OK;
  } catch (const std::bad_alloc&) {
    return fail(c, CLBM_ENOMEM, "host allocation failed");
  }
}

clbm_status clbm_residual(clbm_ctx* c, double* r_out) {
  if (!c || !r_out) return fail(c, CLBM_EINVAL, "bad residual arguments");
  if (c->t < 1) return fail(c, CLBM_EINVAL, "residual needs one step after initialisation");
  const long long n = (long long)c->p.nx * c->p.ny;
  const int nb = red_blocks(n);
  double* out = c->d_part + kMaxRedBlocks * 8;
  CLBM_CUDA(c, c->L->residual(make_geom(c), make_coef(c), c->buf[c->cur], c->buf[c->cur ^ 1],
                              c->d_part, nb, c->stream));
  CLBM_CUDA(c, launch_reduce_partials(c->d_part, nb, 8, out, c->stream));
  double h[8];
  CLBM_CUDA(c, cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  CLBM_CUDA(c, cudaStreamSynchronize(c->stream));
  if (h[6] != 0.0 || !std::isfinite(h[0] + h[1] + h[2] + h[3] + h[4] + h[5])) {
    *r_out = INFINITY;
    return fail(c, CLBM_EUNSTABLE, "non-finite field values");
  }
  double best = 0.0;
  for (int k = 0; k < 3; ++k) {
    const double v = std::sqrt(h[2 * k]) / std::max(std::sqrt(h[2 * k + 1]), 1e-30);
    best = std::max(best, v);
  }
  *r_out = best;
  return CLBM_OK;
}

clbm_status clbm_totals(clbm_ctx* c, double* out) {
  if (!c || !out) return fail(c, CLBM_EINVAL, "bad totals arguments");
  const long long n = (long long)c->p.nx * c->p.ny;
  const int nb = red_blocks(n);
  double* red = c->d_part + kMaxRedBlocks * 8;
  CLBM_CUDA(c, c->L->totals(make_geom(c), c->buf[c->cur], c->d_part, nb, c->stream));
  CLBM_CUDA(c, launch_reduce_partials(c->d_part, nb, 8, red, c->stream));
  double h[8];
  CLBM_CUDA(c, cudaMemcpyAsync(h, red, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  CLBM_CUDA(c, cudaStreamSynchronize(c->stream));
  // the stored values are deviations from the rest state: f_i = w_i rho0 + d_i,
  // g_j = w_j T0 + h_j (the rest state carries no momentum)
  out[0] = h[4] * c->p.rho0 + h[0];
  out[1] = h[1];
  out[2] = h[2];
  out[3] = h[4] * c->p.T0 + h[3];
  if (h[5] != 0.0 || !std::isfinite(out[0] + out[1] + out[2] + out[3]))
    return fail(c, CLBM_EUNSTABLE, "non-finite field values");
  return CLBM_OK;
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
