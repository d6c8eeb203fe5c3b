// capi.cu -- host side of the C ABI declared in include/snap.h: validation, device memory,
// launch sequencing of the Runge-Kutta stages (Sec. 4.3), CUDA-graph replay, budgets and
// status reporting.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/snap.h"
#include "snap_internal.h"

static_assert(snap::kBcReflect == SNAP_REFLECT && snap::kBcPeriodic == SNAP_PERIODIC &&
                  snap::kBcNoSlip == SNAP_NOSLIP && snap::kBcHalo == SNAP_HALO,
              "boundary kinds of the kernels and of the C interface differ");

namespace snap {
bool find_kernels_dry2d(int f32, int visc, KernelSet *out);
bool find_kernels_dry3d(int f32, int visc, KernelSet *out);
bool find_kernels_moist2d(int f32, int visc, int micro, KernelSet *out);
bool find_kernels_moist3d(int f32, int visc, int micro, KernelSet *out);

bool find_adjoint_kernels_dry2d(int f32, AdjKernels *out);
bool find_adjoint_kernels_dry3d(int f32, AdjKernels *out);
bool find_adjoint_kernels_moist2d(int f32, AdjKernels *out);

bool find_adjoint_kernels(int f32, int nvap, int ncond, int three_d, AdjKernels *out) {
  if (nvap == 0) return three_d ? find_adjoint_kernels_dry3d(f32, out) : find_adjoint_kernels_dry2d(f32, out);
  if (nvap == 1 && ncond == 2 && !three_d) return find_adjoint_kernels_moist2d(f32, out);
  return false;
}

bool find_kernels(int f32, int nvap, int ncond, int three_d, int visc, int micro, KernelSet *out) {
  if (nvap == 0 && ncond == 0) return !micro && (three_d ? find_kernels_dry3d(f32, visc, out)
                                                         : find_kernels_dry2d(f32, visc, out));
  if (nvap == 1 && ncond == 2 && !three_d) return find_kernels_moist2d(f32, visc, micro, out);
  if (nvap == 2 && ncond == 2 && three_d) return find_kernels_moist3d(f32, visc, micro, out);
  return false;
}

int budget_blocks(long long ncell) {
  long long b = (ncell + 255) / 256;
  return int(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}

// Caller layout <-> stored layout: the energy field (the last of nv) is shifted by the
// per-level reference e_ref, in FP64; every value is converted to the destination type. One
// grid row per (field, level) plane, so that a block knows its level without dividing the
// element index; VW consecutive elements per thread (one 16-byte access of 4 floats, two of 4
// doubles) where every plane starts on such a boundary, else one.
template <class S, class D, int VW>
__global__ void state_copy_kernel(const S *src, D *dst, int nv, int nz, int k0, long long plane,
                                  const double *e_ref, double sign) {
  const int k = k0 + (int)blockIdx.y, v = blockIdx.z;
  const long long base = ((long long)v * nz + k) * plane;
  const bool shift = e_ref && v == nv - 1;
  const double sh = shift ? sign * e_ref[k] : 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x * VW;
  for (long long q = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * VW; q < plane;
       q += stride) {
    if (VW > 1 && q + VW <= plane) {
      const Pack<S, VW> a = *reinterpret_cast<const Pack<S, VW> *>(src + base + q);
      Pack<D, VW> b;
#pragma unroll
      for (int e = 0; e < VW; ++e) b.x[e] = shift ? D(double(a.x[e]) + sh) : D(a.x[e]);
      *reinterpret_cast<Pack<D, VW> *>(dst + base + q) = b;
    } else {
      for (long long r = q; r < plane && r < q + VW; ++r)
        dst[base + r] = shift ? D(double(src[base + r]) + sh) : D(src[base + r]);
    }
  }
}

template <class S, class D>
static cudaError_t copy_typed(const void *src, void *dst, int nv, long long ncell,
                              long long plane, const double *e_ref, double sg, cudaStream_t s) {
  constexpr int VW = 4;
  const int block = 256;
  const long long nz = ncell / plane;
  const long long per = (plane + (long long)block * VW - 1) / ((long long)block * VW);
  const bool vec = plane % VW == 0 && (uintptr_t)src % (sizeof(S) * VW) == 0 &&
                   (uintptr_t)dst % (sizeof(D) * VW) == 0;
  // levels in chunks of at most 65535 (the grid's y limit); nv is far below the z limit
  for (long long k0 = 0; k0 < nz; k0 += 65535) {
    const long long nk = nz - k0 < 65535 ? nz - k0 : 65535;
    const dim3 grid((unsigned)(per < 4096 ? per : 4096), (unsigned)nk, (unsigned)nv);
    if (vec)
      state_copy_kernel<S, D, VW><<<grid, block, 0, s>>>((const S *)src, (D *)dst, nv, (int)nz,
                                                         (int)k0, plane, e_ref, sg);
    else
      state_copy_kernel<S, D, 1><<<grid, block, 0, s>>>((const S *)src, (D *)dst, nv, (int)nz,
                                                        (int)k0, plane, e_ref, sg);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_state_copy(const void *src, int src_f32, void *dst, int dst_f32, int nv,
                              long long ncell, long long plane, const double *e_ref,
                              int to_stored, cudaStream_t s) {
  const double sg = to_stored ? -1.0 : 1.0;
  if (src_f32 && !dst_f32) return copy_typed<float, double>(src, dst, nv, ncell, plane, e_ref, sg, s);
  if (!src_f32 && dst_f32) return copy_typed<double, float>(src, dst, nv, ncell, plane, e_ref, sg, s);
  if (src_f32) return copy_typed<float, float>(src, dst, nv, ncell, plane, e_ref, sg, s);
  return copy_typed<double, double>(src, dst, nv, ncell, plane, e_ref, sg, s);
}
// The three columns x0 .. x0+2 of every row of a state (fields [nv][nrow][nx]) into a
// contiguous [nv][nrow][3] buffer: a slab's cells next to one of its x sides, which are the
// neighbouring slab's ghost columns. W is an unsigned type of the state's word size (a copy of
// the bits).
template <class W>
__global__ void halo_pack_kernel(const W *Y, W *out, int nv, int nx, long long nrow, int x0) {
  const long long n = (long long)nv * nrow * 3, ncell = nrow * nx;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = int(i % 3);
    const long long r = (i / 3) % nrow, v = i / (3 * nrow);
    out[i] = Y[v * ncell + r * nx + x0 + c];
  }
}
}  // namespace snap

using namespace snap;

struct snap_ctx {
  int ndom = 0;
  int f32 = 0, nvap = 0, ncond = 0, three_d = 0, visc = 0, nv = 0;
  size_t word = 8;
  KernelSet ks{};
  Phys ph{};
  std::vector<snap_grid_desc> desc;
  std::vector<DomDev> dom;   // host mirror of doms_dev
  // slab decomposition: group of each domain (linked slabs share the group's CFL rate and
  // time step slots, rate_dev[grp] and dt_dev[grp]); per domain and x side, 0 = not a halo
  // side or not ready, 1 = linked to a domain of this context, 2 = ghost buffer handed out
  std::vector<int> grp;
  std::vector<int> halo_state;     // [ndom][2]
  void *halo_arena = nullptr;      // ghost buffers of the SNAP_HALO sides
  std::vector<std::vector<double>> rb_host, pf_host;  // reference profiles (host copies)
  std::vector<int> prefix;   // tile prefix per domain
  int ntiles = 0, grid = 0;
  int tv = 0;                // active tile variant
  int persistent = 0;        // 1: one cooperative launch per step (grid barriers between
                             // stages); 2: the resident step (one tile per CTA, neighbour flags)
  int grid_persistent = 0;
  GridSync *gsync = nullptr;
  long long spin_limit = 4000000000ll;  // grid-barrier wait limit, clock cycles (~2 s)
  int absent_cta = -1;                  // test aid (snap_set_barrier_test)
  // resident step: launch bookkeeping, tile flags and ghost-cell dependencies of the current
  // tiling (res_ready: built for tile variant res_tv)
  ResidentSync *res = nullptr;
  unsigned int *tile_flags = nullptr;
  int *dep_begin = nullptr, *dep_list = nullptr;
  unsigned long long *rate_next_dev = nullptr;
  int res_ready = 0, res_tv = -1;
  // size classes (domains of identical nx, ny, nz) and their own tile shapes: with per_class
  // set (three-launch mode only), a stage is one launch per class on parallel streams, each
  // over the class's own tile table (cls_dom, uploaded to cls_doms_dev / cls_prefix_dev)
  std::vector<std::vector<int>> cls;
  std::vector<int> cls_tv, cls_ntiles, cls_off;
  int per_class = 0;
  std::vector<DomDev> cls_dom;
  std::vector<int> cls_prefix;
  DomDev *cls_doms_dev = nullptr;
  int *cls_prefix_dev = nullptr;
  std::vector<cudaStream_t> cls_streams;
  cudaEvent_t ev_fork = nullptr;
  std::vector<cudaEvent_t> ev_join;
  int only_class = -1;  // autotuner: launch this class alone
  // discrete adjoint (dry, inviscid, one domain): recording and work buffers
  int has_adj = 0;
  AdjKernels adj{};
  int rec_steps = 0, ckpt_every = 0;
  std::vector<double> rec_dt;
  void *ckpt = nullptr;       // checkpoints every ckpt_every steps, then the final state
  void *segbuf = nullptr;     // states of one segment, or of two (see snap_step_adjoint)
  int nsegbuf = 1;
  cudaStream_t rec_stream = nullptr;  // recomputation of the next segment
  cudaEvent_t ev_rec[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
  double *dt_hist = nullptr;  // device copy of the recorded time steps
  void *lam = nullptr;        // four adjoint vectors
  void *gface = nullptr;      // per-direction face contributions
  size_t gface_off[3] = {0, 0, 0};
  void *adjw = nullptr;       // FP64 adjoint: primitives and per-direction window results
  size_t adjw_off[4] = {0, 0, 0, 0};
  // device memory
  void *arena = nullptr;
  DomDev *doms_dev = nullptr;
  int *prefix_dev = nullptr;
  double *prof_dev = nullptr;
  float *proff_dev = nullptr;
  unsigned long long *rate_dev = nullptr;
  double *dt_dev = nullptr;
  unsigned int *flags_dev = nullptr;
  int *sweeps_dev = nullptr;
  double *budget_partials = nullptr;
  double *budget_out = nullptr;
  void *staging = nullptr;
  size_t staging_bytes = 0;
  long long state_bytes = 0, ncells = 0;
  // execution
  cudaStream_t own_stream = nullptr, stream = nullptr;
  int use_graph = 1;
  cudaGraphExec_t graph = nullptr;
  double graph_dt = -1.0;
  std::string err;
};

static thread_local std::string g_init_error;

static int fail(snap_ctx *c, int code, const std::string &msg) {
  if (c)
    c->err = msg;
  else
    g_init_error = msg;
  return code;
}

static int cuda_fail(snap_ctx *c, cudaError_t e, const char *where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return fail(c, SNAP_ENOMEM, m);
  return fail(c, SNAP_ECUDA, m);
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);  \
  } while (0)

static void release(snap_ctx *ctx) {
  if (!ctx) return;
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  cudaFree(ctx->arena);
  cudaFree(ctx->halo_arena);
  cudaFree(ctx->doms_dev);
  cudaFree(ctx->prefix_dev);
  cudaFree(ctx->gsync);
  cudaFree(ctx->res);
  cudaFree(ctx->tile_flags);
  cudaFree(ctx->dep_begin);
  cudaFree(ctx->dep_list);
  cudaFree(ctx->rate_next_dev);
  cudaFree(ctx->cls_doms_dev);
  cudaFree(ctx->cls_prefix_dev);
  for (cudaStream_t st : ctx->cls_streams) cudaStreamDestroy(st);
  for (cudaEvent_t ev : ctx->ev_join) cudaEventDestroy(ev);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  cudaFree(ctx->ckpt);
  cudaFree(ctx->segbuf);
  if (ctx->rec_stream) cudaStreamDestroy(ctx->rec_stream);
  for (int b = 0; b < 2; ++b) {
    if (ctx->ev_rec[b]) cudaEventDestroy(ctx->ev_rec[b]);
    if (ctx->ev_free[b]) cudaEventDestroy(ctx->ev_free[b]);
  }
  cudaFree(ctx->dt_hist);
  cudaFree(ctx->lam);
  cudaFree(ctx->gface);
  cudaFree(ctx->adjw);
  cudaFree(ctx->prof_dev);
  cudaFree(ctx->proff_dev);
  cudaFree(ctx->rate_dev);
  cudaFree(ctx->dt_dev);
  cudaFree(ctx->flags_dev);
  cudaFree(ctx->sweeps_dev);
  cudaFree(ctx->budget_partials);
  cudaFree(ctx->budget_out);
  cudaFree(ctx->staging);
  if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
}

static int validate(const snap_grid_desc &d, const snap_grid_desc &d0, int idx, std::string &m) {
  char b[256];
  auto bad = [&](const char *what) {
    snprintf(b, sizeof b, "domain %d: %s", idx, what);
    m = b;
    return SNAP_EINVAL;
  };
  if (d.nx < 3 || d.nz < 3 || d.ny < 1 || d.ny == 2) return bad("need nx >= 3, nz >= 3, ny == 1 or ny >= 3");
  if (!(d.dx > 0) || !(d.dz > 0) || (d.ny > 1 && !(d.dy > 0))) return bad("cell sizes must be positive");
  for (int s = 0; s < 6; ++s)
    if (d.bc[s] != SNAP_REFLECT && d.bc[s] != SNAP_PERIODIC && d.bc[s] != SNAP_NOSLIP &&
        !(d.bc[s] == SNAP_HALO && s < 2))
      return bad("bc must be REFLECT, PERIODIC or NOSLIP (or HALO on an x side)");
  if (d.bc[4] == SNAP_PERIODIC || d.bc[5] == SNAP_PERIODIC) return bad("the z boundaries must be walls");
  if (!isfinite(d.T_bottom) || !(d.T_bottom >= 0.0)) return bad("T_bottom must be finite and >= 0");
  if ((d.bc[0] == SNAP_PERIODIC) != (d.bc[1] == SNAP_PERIODIC)) return bad("periodic x needs both x sides periodic");
  if ((d.bc[2] == SNAP_PERIODIC) != (d.bc[3] == SNAP_PERIODIC)) return bad("periodic y needs both y sides periodic");
  if (!(d.gamma_d > 1.0) || !(d.R_d > 0.0)) return bad("gamma_d > 1 and R_d > 0 required");
  if (!(d.grav >= 0.0)) return bad("grav must be >= 0");
  if (!(d.cfl > 0.0)) return bad("cfl must be > 0");
  if (!(d.weno_eps > 0.0)) return bad("weno_eps must be > 0");
  if (d.n_vapor < 0 || d.n_vapor > SNAP_MAX_VAPOR) return bad("n_vapor out of range");
  if (d.n_cond < 0 || d.n_cond > SNAP_MAX_COND) return bad("n_cond out of range");
  if (d.dtype != SNAP_F64 && d.dtype != SNAP_F32) return bad("dtype must be SNAP_F64 or SNAP_F32");
  if (d.satadj && (d.n_vapor == 0 || d.n_cond == 0)) return bad("satadj needs vapours with condensates");
  if (d.satadj && d.satadj_max_iter < 1) return bad("satadj_max_iter must be >= 1");
  if (!(d.nu >= 0.0)) return bad("nu must be >= 0");
  for (int j = 0; j < SNAP_MAX_COND; ++j)
    if (!isfinite(d.w_term[j]) || (d.w_term[j] != 0.0 && j >= d.n_cond))
      return bad("w_term must be finite and zero beyond n_cond");
  if (!isfinite(d.cool_rate) || !(d.sponge_tau0 >= 0.0) || (d.sponge_tau0 > 0.0 && !(d.sponge_p0 > 0.0)))
    return bad("cooling rate must be finite, sponge_tau0 >= 0 with sponge_p0 > 0");
  if ((d.cool_rate != 0.0 || d.sponge_tau0 > 0.0) && d.n_vapor < 1)
    return bad("the forcing is built for moist contexts (n_vapor > 0)");
  if (d.kessler) {
    if (d.n_vapor < 1 || d.n_cond != 2) return bad("the Kessler scheme needs vapours with cloud and precipitation (n_cond == 2)");
    if (d.kessler_max_iter < 1) return bad("kessler_max_iter must be >= 1");
    for (int r = 0; r < 4; ++r)
      if (!(d.kessler_k[r] >= 0.0)) return bad("Kessler rates must be >= 0");
  }
  if (!d.rho_bar || !d.p_bar_face) return bad("reference profile pointers are NULL");
  for (int k = 0; k < d.nz; ++k) {
    if (!(d.rho_bar[k] > 0) || !(d.p_bar_face[k] > 0) || !(d.p_bar_face[k + 1] > 0))
      return bad("reference profile must be positive");
    double want = d.p_bar_face[k] - d.grav * d.rho_bar[k] * d.dz;
    if (fabs(d.p_bar_face[k + 1] - want) > 1e-9 * d.p_bar_face[k])
      return bad("reference profile is not discretely hydrostatic");
  }
  if (d.dtype != d0.dtype || d.n_vapor != d0.n_vapor || d.n_cond != d0.n_cond ||
      (d.ny > 1) != (d0.ny > 1) || d.gamma_d != d0.gamma_d || d.R_d != d0.R_d ||
      (d.nu > 0) != (d0.nu > 0) || d.nu != d0.nu || d.satadj != d0.satadj ||
      d.weno_eps != d0.weno_eps || d.kessler != d0.kessler ||
      memcmp(d.kessler_k, d0.kessler_k, sizeof d.kessler_k) != 0 ||
      memcmp(d.w_term, d0.w_term, sizeof d.w_term) != 0 || d.cool_rate != d0.cool_rate ||
      d.cool_p_lo != d0.cool_p_lo || d.cool_p_hi != d0.cool_p_hi ||
      d.sponge_tau0 != d0.sponge_tau0 || d.sponge_p0 != d0.sponge_p0)
    return bad("domains of one context must share dtype, species, gases, dimensionality, "
               "viscosity and scheme options");
  for (int i = 0; i < d.n_vapor; ++i) {
    const snap_species &s = d.species[i], &s0 = d0.species[i];
    if (!(s.eps > 0) || !(s.sigma_v > 0) || !(s.T_ref > 0) || !(s.p_ref > 0))
      return bad("species constants must be positive");
    if (memcmp(&s, &s0, sizeof s) != 0) return bad("domains must share the species table");
  }
  return SNAP_OK;
}

static void derive_phys(const snap_grid_desc &d, Phys &ph) {
  memset(&ph, 0, sizeof ph);
  ph.gamma_d = d.gamma_d;
  ph.R_d = d.R_d;
  ph.c_vd = d.R_d / (d.gamma_d - 1.0);
  ph.c_pd = d.gamma_d * ph.c_vd;
  ph.kappa = d.R_d / ph.c_pd;
  ph.nvap = d.n_vapor;
  ph.ncond = d.n_cond;
  for (int i = 0; i < d.n_vapor; ++i) {
    const snap_species &s = d.species[i];
    ph.eps[i] = s.eps;
    ph.inv_eps[i] = 1.0 / s.eps;
    ph.sig_v[i] = s.sigma_v;
    ph.R_v[i] = d.R_d / s.eps;
    ph.sig_hat[i] = s.sigma_v * s.eps;
    ph.Tref[i] = s.T_ref;
    ph.pref[i] = s.p_ref;
    const double c_pv = s.sigma_v * ph.c_vd + ph.R_v[i];
    for (int j = 0; j < d.n_cond; ++j) {
      ph.sig_c[i][j] = s.sigma_c[j];
      const double dc = s.sigma_c[j] * ph.c_vd - c_pv;   // Eq. latent
      ph.mu[i][j] = -(s.L_ref[j] + dc * s.T_ref);         // Eq. muij with mu_i = 0
    }
    if (d.n_cond > 0) {
      const double dc = s.sigma_c[0] * ph.c_vd - c_pv;
      ph.beta[i] = (s.L_ref[0] + dc * s.T_ref) / (ph.R_v[i] * s.T_ref);  // App. D
      ph.delta[i] = dc / ph.R_v[i];
    }
  }
  ph.weno_eps = d.weno_eps;
  ph.nu = d.nu;
  ph.satadj = d.satadj;
  ph.satadj_max_iter = d.satadj_max_iter;
  ph.satadj_tol = d.satadj_tol;
  ph.sediment = 0;
  for (int j = 0; j < kMaxCond; ++j) {
    ph.w_term[j] = j < d.n_cond ? d.w_term[j] : 0.0;
    if (ph.w_term[j] != 0.0) ph.sediment = 1;
  }
  ph.kessler = d.kessler;
  ph.kessler_max_iter = d.kessler_max_iter;
  ph.kessler_tol = d.kessler_tol;
  for (int r = 0; r < 4; ++r) ph.kessler_k[r] = d.kessler_k[r];
  ph.cool_rate = d.cool_rate;
  ph.cool_p_lo = d.cool_p_lo;
  ph.cool_p_hi = d.cool_p_hi;
  ph.sponge_tau0 = d.sponge_tau0;
  ph.sponge_p0 = d.sponge_p0;
}

template <class T>
static void derive_cst(const Phys &ph, double tol_floor, CstT<T> &c) {
  memset(&c, 0, sizeof c);
  c.gamma_d = T(ph.gamma_d);
  c.gm1 = T(ph.gamma_d - 1.0);
  c.igm1 = T(1.0 / (ph.gamma_d - 1.0));
  c.R_d = T(ph.R_d);
  c.iR_d = T(1.0 / ph.R_d);
  c.kappa = T(ph.kappa);
  c.c_pd = T(ph.c_pd);
  c.nu = T(ph.nu);
  c.weno_eps = T(ph.weno_eps);
  c.satadj_tol = T(ph.satadj_tol > tol_floor ? ph.satadj_tol : tol_floor);
  for (int i = 0; i < kMaxVap; ++i) {
    c.eps[i] = T(ph.eps[i]);
    c.inv_eps[i] = T(ph.inv_eps[i]);
    c.ieps_m1[i] = T(ph.inv_eps[i] - 1.0);
    c.sig_v[i] = T(ph.sig_v[i]);
    c.sigv_m1[i] = T(ph.sig_v[i] - 1.0);
    c.pref[i] = T(ph.pref[i]);
    c.beta[i] = T(ph.beta[i]);
    c.delta[i] = T(ph.delta[i]);
    c.inv_Tref[i] = T(ph.Tref[i] > 0 ? 1.0 / ph.Tref[i] : 0.0);
    c.sighat_m1[i] = T(ph.sig_hat[i] - 1.0);
    for (int j = 0; j < kMaxCond; ++j) {
      c.sig_c[i][j] = T(ph.sig_c[i][j]);
      c.sigc_m1[i][j] = T(ph.sig_c[i][j] - 1.0);
      c.mu[i][j] = T(ph.mu[i][j]);
    }
  }
  for (int j = 0; j < kMaxCond; ++j) c.w_term[j] = T(ph.w_term[j]);
  for (int r = 0; r < 4; ++r) c.kk[r] = T(ph.kessler_k[r]);
  c.kessler_tol = T(ph.kessler_tol > tol_floor ? ph.kessler_tol : tol_floor);
  c.c_vd = T(ph.c_vd);
  c.cool_rate = T(ph.cool_rate);
  c.cool_p_lo = T(ph.cool_p_lo);
  c.cool_p_hi = T(ph.cool_p_hi);
  c.sponge_itau0 = T(ph.sponge_tau0 > 0 ? 1.0 / ph.sponge_tau0 : 0.0);
  c.sponge_ip0 = T(ph.sponge_p0 > 0 ? 1.0 / ph.sponge_p0 : 0.0);
}

static StageArgs args_of(snap_ctx *ctx, int stage) {
  StageArgs a;
  a.doms = ctx->doms_dev;
  a.tile_domain = ctx->prefix_dev;
  a.ndom = ctx->ndom;
  a.ntiles = ctx->ntiles;
  a.stage = stage;
  a.flags = ctx->flags_dev;
  a.max_sweeps = ctx->sweeps_dev;
  a.gsync = ctx->gsync;
  a.spin_limit = ctx->spin_limit;
  a.absent_cta = ctx->absent_cta;
  a.res = ctx->res;
  a.tile_flags = ctx->tile_flags;
  a.dep_begin = ctx->dep_begin;
  a.dep_list = ctx->dep_list;
  a.dt_override = -1.0;
  a.buf_s = a.buf_n = nullptr;
  a.buf_o = nullptr;
  a.ph = ctx->ph;
  // stop tolerance of the adjustment: at least 32 machine epsilons of the arithmetic type
  derive_cst<float>(ctx->ph, 32.0 * 1.1920928955078125e-07, a.cf);
  derive_cst<double>(ctx->ph, 32.0 * 2.220446049250313e-16, a.cd);
  return a;
}

// CFL rate of the group of domain dm (the domain itself unless it is a linked slab): the
// group's slot is cleared and every member's cells take their maximum into it.
static int refresh_rate(snap_ctx *ctx, int dm, cudaStream_t s) {
  const int g = ctx->grp[dm];
  CK(cudaMemsetAsync(ctx->rate_dev + g, 0, sizeof(unsigned long long), s));
  StageArgs a = args_of(ctx, 0);
  for (int i = 0; i < ctx->ndom; ++i)
    if (ctx->grp[i] == g) CK(ctx->ks.rate(a, i, 0, s));
  return SNAP_OK;
}

// Every SNAP_HALO side linked or its ghost buffer handed out.
static int halos_ready(snap_ctx *ctx, const char *who) {
  for (int i = 0; i < ctx->ndom; ++i)
    for (int h = 0; h < 2; ++h)
      if (ctx->dom[i].bc[h] == kBcHalo && ctx->halo_state[2 * i + h] == 0)
        return fail(ctx, SNAP_EINVAL, std::string(who) + ": a SNAP_HALO side is neither linked "
                                      "(snap_link_halo) nor fed (snap_halo_buffer)");
  return SNAP_OK;
}

static int apply_variant(snap_ctx *ctx, int v);
static int build_class_tables(snap_ctx *ctx);

// Default tile shape: the first variant (in the order built, the fastest on large grids) whose
// tiles over all domains fill every SM at least once; else the one with the most tiles.
static int default_variant(const snap_ctx *ctx) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  int best = 0;
  long long best_tiles = -1;
  for (int v = 0; v < ctx->ks.nvariants; ++v) {
    const int *tl = ctx->ks.var[v].tile;
    long long t = 0;
    for (const DomDev &D : ctx->dom)
      t += (long long)((D.nx + tl[0] - 1) / tl[0]) * ((D.ny + tl[1] - 1) / tl[1]) *
           ((D.nz + tl[2] - 1) / tl[2]);
    if (t >= nsm) return v;
    if (t > best_tiles) {
      best_tiles = t;
      best = v;
    }
  }
  return best;
}

extern "C" int snap_init_grid(snap_ctx **out, const snap_grid_desc *d, int n_domains) {
  snap_ctx *ctx = nullptr;
  if (!out || !d || n_domains < 1) return fail(nullptr, SNAP_EINVAL, "snap_init_grid: bad arguments");
  *out = nullptr;
  std::string m;
  for (int i = 0; i < n_domains; ++i) {
    int rc = validate(d[i], d[0], i, m);
    if (rc) return fail(nullptr, rc, m);
  }
  ctx = new (std::nothrow) snap_ctx();
  if (!ctx) return fail(nullptr, SNAP_ENOMEM, "snap_init_grid: host allocation failed");
  ctx->ndom = n_domains;
  ctx->f32 = d[0].dtype == SNAP_F32;
  ctx->nvap = d[0].n_vapor;
  ctx->ncond = d[0].n_cond;
  ctx->three_d = d[0].ny > 1;
  ctx->visc = d[0].nu > 0.0;
  ctx->nv = 1 + ctx->nvap + ctx->nvap * ctx->ncond + (ctx->three_d ? 3 : 2) + 1;
  ctx->word = ctx->f32 ? 4 : 8;
  // microphysics, sedimentation or forcing pick kernels with those terms compiled in
  int micro = d[0].kessler != 0 || d[0].cool_rate != 0.0 || d[0].sponge_tau0 > 0.0;
  for (int j = 0; j < SNAP_MAX_COND; ++j) micro |= d[0].w_term[j] != 0.0;
  if (!find_kernels(ctx->f32, ctx->nvap, ctx->ncond, ctx->three_d, ctx->visc, micro, &ctx->ks)) {
    delete ctx;
    return fail(nullptr, SNAP_ENOTSUP,
                "snap_init_grid: this library builds dry (any dimension, optional viscosity), "
                "one vapour with two condensates (x-z plane) and two vapours with two "
                "condensates (3-D) without viscosity");
  }
  derive_phys(d[0], ctx->ph);
  ctx->desc.assign(d, d + n_domains);
  // the adjoint covers neither the microphysics nor sedimentation, nor no-slip walls or a
  // fixed bottom temperature
  bool plain_walls = d[0].T_bottom == 0.0;
  for (int s = 0; s < 6; ++s)
    plain_walls = plain_walls && d[0].bc[s] != SNAP_NOSLIP && d[0].bc[s] != SNAP_HALO;
  if (!ctx->visc && n_domains == 1 && !micro && plain_walls)
    ctx->has_adj = find_adjoint_kernels(ctx->f32, ctx->nvap, ctx->ncond, ctx->three_d, &ctx->adj) ? 1 : 0;
  cudaError_t e = cudaSuccess;
  for (int v = 0; v < ctx->ks.nvariants && e == cudaSuccess; ++v) e = ctx->ks.var[v].prepare();
  if (e != cudaSuccess) {
    int rc = cuda_fail(nullptr, e, "snap_init_grid: kernel attributes");
    delete ctx;
    return rc;
  }
  // layout of the state arena and tile table
  std::vector<size_t> off(n_domains);
  size_t total = 0, maxcell = 0;
  size_t nprof = 0, nproff = 0;
  ctx->prefix.assign(n_domains + 1, 0);
  ctx->dom.resize(n_domains);
  ctx->grp.resize(n_domains);
  ctx->halo_state.assign(2 * (size_t)n_domains, 0);
  ctx->rb_host.resize(n_domains);
  ctx->pf_host.resize(n_domains);
  std::vector<size_t> halo_off(2 * (size_t)n_domains, 0);
  size_t halo_total = 0;
  for (int i = 0; i < n_domains; ++i) {
    const snap_grid_desc &g = d[i];
    size_t nc = (size_t)g.nx * g.ny * g.nz;
    size_t bytes = ((nc * ctx->nv * ctx->word) + 255) / 256 * 256;
    off[i] = total;
    total += 3 * bytes;
    maxcell = nc > maxcell ? nc : maxcell;
    ctx->ncells += (long long)nc;
    ctx->state_bytes += (long long)(nc * ctx->nv * ctx->word);
    nprof += 4 * (size_t)g.nz + 1;
    nproff += 5 * (size_t)g.nz + 1;
    DomDev &D = ctx->dom[i];
    D.nx = g.nx;
    D.ny = g.ny;
    D.nz = g.nz;
    const int *tl = ctx->ks.var[0].tile;
    D.tx = (g.nx + tl[0] - 1) / tl[0];
    D.ty = (g.ny + tl[1] - 1) / tl[1];
    D.tz = (g.nz + tl[2] - 1) / tl[2];
    D.tile_begin = ctx->prefix[i];
    ctx->prefix[i + 1] = ctx->prefix[i] + D.tx * D.ty * D.tz;
    for (int s = 0; s < 6; ++s) D.bc[s] = g.bc[s];
    D.dx = g.dx;
    D.dy = g.ny > 1 ? g.dy : g.dx;
    D.dz = g.dz;
    D.grav = g.grav;
    D.cfl = g.cfl;
    D.dt_fixed = -1.0;
    D.T_bot = g.T_bottom;
    D.ncell = (long long)nc;
    (void)bytes;
    ctx->grp[i] = i;
    ctx->rb_host[i].assign(g.rho_bar, g.rho_bar + g.nz);
    ctx->pf_host[i].assign(g.p_bar_face, g.p_bar_face + g.nz + 1);
    for (int h = 0; h < 2; ++h) {
      D.hnx[h] = 3;
      D.hoff[h] = 0;
      for (int st = 0; st < 3; ++st) D.hsrc[h][st] = nullptr;
      if (g.bc[h] == SNAP_HALO) {
        halo_off[2 * i + h] = halo_total;
        halo_total += ((size_t)ctx->nv * g.nz * g.ny * 3 * ctx->word + 255) / 256 * 256;
      }
    }
  }
  ctx->ntiles = ctx->prefix[n_domains];
  int ret = SNAP_OK;
  do {
    ctx->grid = ctx->ntiles;
    if ((e = cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking)) != cudaSuccess) break;
    ctx->stream = ctx->own_stream;
    if ((e = cudaMalloc(&ctx->arena, total)) != cudaSuccess) break;
    if ((e = cudaMemset(ctx->arena, 0, total)) != cudaSuccess) break;
    if (halo_total) {
      if ((e = cudaMalloc(&ctx->halo_arena, halo_total)) != cudaSuccess) break;
      if ((e = cudaMemset(ctx->halo_arena, 0, halo_total)) != cudaSuccess) break;
      for (int i = 0; i < n_domains; ++i)
        for (int h = 0; h < 2; ++h)
          if (d[i].bc[h] == SNAP_HALO)
            for (int st = 0; st < 3; ++st)
              ctx->dom[i].hsrc[h][st] = (char *)ctx->halo_arena + halo_off[2 * i + h];
    }
    if ((e = cudaMalloc(&ctx->doms_dev, sizeof(DomDev) * n_domains)) != cudaSuccess) break;
    if ((e = cudaMalloc(&ctx->prefix_dev, sizeof(int) * (n_domains + 1))) != cudaSuccess) break;
    if ((e = cudaMalloc(&ctx->gsync, sizeof(GridSync))) != cudaSuccess) break;
    if ((e = cudaMemset(ctx->gsync, 0, sizeof(GridSync))) != cudaSuccess) break;
    if ((e = cudaMalloc(&ctx->prof_dev, sizeof(double) * nprof)) != cudaSuccess) break;
    if ((e = cudaMalloc(&ctx->proff_dev, sizeof(float) * nproff)) != cudaSuccess) break;
    if ((e = cudaMalloc(&ctx->rate_dev, sizeof(unsigned long long) * n_domains)) != cudaSuccess) break;
    if ((e = cudaMalloc(&ctx->rate_next_dev, sizeof(unsigned long long) * n_domains)) != cudaSuccess) break;
    if ((e = cudaMemset(ctx->rate_next_dev, 0, sizeof(unsigned long long) * n_domains)) != cudaSuccess) break;
    if ((e = cudaMalloc(&ctx->res, sizeof(ResidentSync))) != cudaSuccess) break;
    if ((e = cudaMalloc(&ctx->dt_dev, sizeof(double) * n_domains)) != cudaSuccess) break;
    if ((e = cudaMalloc(&ctx->flags_dev, sizeof(unsigned int))) != cudaSuccess) break;
    if ((e = cudaMalloc(&ctx->sweeps_dev, sizeof(int))) != cudaSuccess) break;
    if ((e = cudaMalloc(&ctx->budget_partials, sizeof(double) * 1024 * (ctx->nv + 1))) != cudaSuccess) break;
    if ((e = cudaMalloc(&ctx->budget_out, sizeof(double) * (ctx->nv + 1))) != cudaSuccess) break;
    ctx->staging_bytes = maxcell * ctx->nv * 8;
    if ((e = cudaMalloc(&ctx->staging, ctx->staging_bytes)) != cudaSuccess) break;
    if ((e = cudaMemset(ctx->rate_dev, 0, sizeof(unsigned long long) * n_domains)) != cudaSuccess) break;
    if ((e = cudaMemset(ctx->dt_dev, 0, sizeof(double) * n_domains)) != cudaSuccess) break;
    if ((e = cudaMemset(ctx->flags_dev, 0, sizeof(unsigned int))) != cudaSuccess) break;
    if ((e = cudaMemset(ctx->sweeps_dev, 0, sizeof(int))) != cudaSuccess) break;
    std::vector<double> prof(nprof);
    std::vector<float> proff(nproff);
    size_t po = 0, pof = 0;
    for (int i = 0; i < n_domains; ++i) {
      const snap_grid_desc &g = d[i];
      DomDev &D = ctx->dom[i];
      size_t nc = (size_t)g.nx * g.ny * g.nz;
      size_t bytes = ((nc * ctx->nv * ctx->word) + 255) / 256 * 256;
      for (int b = 0; b < 3; ++b) D.buf[b] = (char *)ctx->arena + off[i] + b * bytes;
      double *rb = ctx->prof_dev + po, *pf = rb + g.nz, *pc = pf + g.nz + 1, *er = pc + g.nz;
      for (int k = 0; k < g.nz; ++k) {
        const double pk = 0.5 * (g.p_bar_face[k] + g.p_bar_face[k + 1]);
        prof[po + k] = g.rho_bar[k];
        prof[po + 2 * g.nz + 1 + k] = pk;
        prof[po + 3 * g.nz + 1 + k] = pk / (g.gamma_d - 1.0);
      }
      for (int k = 0; k <= g.nz; ++k) prof[po + g.nz + k] = g.p_bar_face[k];
      D.rho_bar = rb;
      D.p_face = pf;
      D.p_cell = pc;
      D.e_ref = er;
      // FP32 copies: rho_bar as hi + lo, reference pressures and energies rounded
      float *fb = ctx->proff_dev + pof;
      for (int k = 0; k < g.nz; ++k) {
        const float hi = (float)g.rho_bar[k];
        proff[pof + k] = hi;
        proff[pof + g.nz + k] = (float)(g.rho_bar[k] - (double)hi);
        proff[pof + 2 * g.nz + k] = (float)prof[po + 2 * g.nz + 1 + k];
        proff[pof + 4 * g.nz + 1 + k] = (float)prof[po + 3 * g.nz + 1 + k];
      }
      for (int k = 0; k <= g.nz; ++k) proff[pof + 3 * g.nz + k] = (float)g.p_bar_face[k];
      D.rb_hi = fb;
      D.rb_lo = fb + g.nz;
      D.pc_f = fb + 2 * g.nz;
      D.pf_f = fb + 3 * g.nz;
      D.er_f = fb + 4 * g.nz + 1;
      D.idx = 1.0 / D.dx;
      D.idy = 1.0 / D.dy;
      D.idz = 1.0 / D.dz;
      D.fidx = (float)D.idx;
      D.fidy = (float)D.idy;
      D.fidz = (float)D.idz;
      D.fgrav = (float)g.grav;
      D.rate = ctx->rate_dev + i;
      D.rate_next = ctx->rate_next_dev + i;
      D.dt_step = ctx->dt_dev + i;
      po += 4 * (size_t)g.nz + 1;
      pof += 5 * (size_t)g.nz + 1;
    }
    if ((e = cudaMemcpy(ctx->prof_dev, prof.data(), sizeof(double) * nprof, cudaMemcpyHostToDevice)) != cudaSuccess) break;
    if ((e = cudaMemcpy(ctx->proff_dev, proff.data(), sizeof(float) * nproff, cudaMemcpyHostToDevice)) != cudaSuccess) break;
    if ((e = cudaMemcpy(ctx->doms_dev, ctx->dom.data(), sizeof(DomDev) * n_domains, cudaMemcpyHostToDevice)) != cudaSuccess) break;
    if ((e = cudaMemcpy(ctx->prefix_dev, ctx->prefix.data(), sizeof(int) * (n_domains + 1), cudaMemcpyHostToDevice)) != cudaSuccess) break;
  } while (0);
  if (e != cudaSuccess) {
    ret = cuda_fail(nullptr, e, "snap_init_grid");
    release(ctx);
    delete ctx;
    return ret;
  }
  {
    int mrb = ctx->ks.var[0].max_resident_blocks();
    ctx->grid_persistent = mrb < ctx->ntiles ? mrb : ctx->ntiles;
  }
  for (int i = 0; i < n_domains; ++i) {
    int c = 0;
    while (c < (int)ctx->cls.size()) {
      const DomDev &A = ctx->dom[ctx->cls[c][0]];
      if (A.nx == ctx->dom[i].nx && A.ny == ctx->dom[i].ny && A.nz == ctx->dom[i].nz) break;
      ++c;
    }
    if (c == (int)ctx->cls.size()) ctx->cls.emplace_back();
    ctx->cls[c].push_back(i);
  }
  ctx->cls_tv.assign(ctx->cls.size(), 0);
  ctx->cls_ntiles.assign(ctx->cls.size(), 0);
  if (const int v = default_variant(ctx)) {
    if ((ret = apply_variant(ctx, v)) != SNAP_OK) {
      g_init_error = "snap_init_grid: " + ctx->err;
      release(ctx);
      delete ctx;
      return ret;
    }
  }
  *out = ctx;
  return SNAP_OK;
}

// Rebuild the tile tables of every domain for tile variant v and upload them.
static int apply_variant(snap_ctx *ctx, int v) {
  const int *tl = ctx->ks.var[v].tile;
  ctx->prefix[0] = 0;
  for (int i = 0; i < ctx->ndom; ++i) {
    DomDev &D = ctx->dom[i];
    D.tx = (D.nx + tl[0] - 1) / tl[0];
    D.ty = (D.ny + tl[1] - 1) / tl[1];
    D.tz = (D.nz + tl[2] - 1) / tl[2];
    D.tile_begin = ctx->prefix[i];
    ctx->prefix[i + 1] = ctx->prefix[i] + D.tx * D.ty * D.tz;
  }
  ctx->ntiles = ctx->prefix[ctx->ndom];
  ctx->grid = ctx->ntiles;
  const int mrb = ctx->ks.var[v].max_resident_blocks();
  if (mrb <= 0) return fail(ctx, SNAP_ECUDA, "occupancy query of the step kernel failed");
  ctx->grid_persistent = mrb < ctx->ntiles ? mrb : ctx->ntiles;
  ctx->tv = v;
  ctx->res_ready = 0;
  for (int &t : ctx->cls_tv) t = v;
  ctx->per_class = 0;
  CK(cudaMemcpyAsync(ctx->doms_dev, ctx->dom.data(), sizeof(DomDev) * ctx->ndom,
                     cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->prefix_dev, ctx->prefix.data(), sizeof(int) * (ctx->ndom + 1),
                     cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->graph) {
    cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
  }
  return SNAP_OK;
}

static cudaStream_t pick(snap_ctx *ctx, void *stream) {
  return stream ? (cudaStream_t)stream : ctx->stream;  // NULL: the context's current stream
}

// Device address of page-locked host memory (a pinned buffer is mapped into the device's
// address space): the conversion kernel then reads or writes it directly over the host link,
// with no staging copy. nullptr for pageable memory.
static void *mapped_host(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) == cudaSuccess && a.type == cudaMemoryTypeHost &&
      a.devicePointer)
    return a.devicePointer;
  cudaGetLastError();
  return nullptr;
}

extern "C" int snap_set_state(snap_ctx *ctx, int domain, const void *Y, int dtype, int on_device,
                              void *stream) {
  if (!ctx) return fail(nullptr, SNAP_EINVAL, "snap_set_state: NULL context");
  if (domain < 0 || domain >= ctx->ndom || !Y || (dtype != SNAP_F64 && dtype != SNAP_F32))
    return fail(ctx, SNAP_EINVAL, "snap_set_state: bad domain, pointer or dtype");
  cudaStream_t s = pick(ctx, stream);
  const DomDev &D = ctx->dom[domain];
  const long long n = D.ncell * ctx->nv;
  const int src_f32 = dtype == SNAP_F32;
  const size_t sw = src_f32 ? 4 : 8;
  const void *src = Y;
  if (!on_device) {
    if (const void *m = mapped_host(Y)) {
      src = m;
    } else {
      CK(cudaMemcpyAsync(ctx->staging, Y, n * sw, cudaMemcpyHostToDevice, s));
      src = ctx->staging;
    }
  }
  // the stored state and its CFL rate in one pass; the rate slot is shared by the domains of
  // a CFL group, so the others' rates are formed again after it is cleared
  const int g = ctx->grp[domain];
  CK(cudaMemsetAsync(ctx->rate_dev + g, 0, sizeof(unsigned long long), s));
  const StageArgs a = args_of(ctx, 0);
  CK(ctx->ks.load(src, src_f32, a, domain, (long long)D.nx * D.ny, D.nz, s));
  for (int i = 0; i < ctx->ndom; ++i)
    if (i != domain && ctx->grp[i] == g) CK(ctx->ks.rate(a, i, 0, s));
  return SNAP_OK;
}

extern "C" int snap_get_state(snap_ctx *ctx, int domain, void *Y_out, int dtype, int on_device,
                              void *stream) {
  if (!ctx) return fail(nullptr, SNAP_EINVAL, "snap_get_state: NULL context");
  if (domain < 0 || domain >= ctx->ndom || !Y_out || (dtype != SNAP_F64 && dtype != SNAP_F32))
    return fail(ctx, SNAP_EINVAL, "snap_get_state: bad domain, pointer or dtype");
  cudaStream_t s = pick(ctx, stream);
  const DomDev &D = ctx->dom[domain];
  const long long n = D.ncell * ctx->nv;
  const int dst_f32 = dtype == SNAP_F32;
  const size_t dw = dst_f32 ? 4 : 8;
  void *mapped = on_device ? nullptr : mapped_host(Y_out);
  void *dst = on_device ? Y_out : (mapped ? mapped : ctx->staging);
  CK(launch_state_copy(D.buf[0], ctx->f32, dst, dst_f32, ctx->nv, D.ncell,
                       (long long)D.nx * D.ny, D.e_ref, 0, s));
  if (!on_device) {
    if (!mapped) CK(cudaMemcpyAsync(Y_out, ctx->staging, n * dw, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  return SNAP_OK;
}

static int set_dt_fixed(snap_ctx *ctx, double dt_fixed) {
  bool changed = false;
  for (int i = 0; i < ctx->ndom; ++i) {
    double want = dt_fixed > 0.0 ? dt_fixed : -1.0;
    if (ctx->dom[i].dt_fixed != want) {
      ctx->dom[i].dt_fixed = want;
      changed = true;
    }
  }
  if (changed) {
    CK(cudaMemcpyAsync(ctx->doms_dev, ctx->dom.data(), sizeof(DomDev) * ctx->ndom,
                       cudaMemcpyHostToDevice, ctx->stream));
    if (ctx->per_class || ctx->only_class >= 0) return build_class_tables(ctx);
  }
  return SNAP_OK;
}

// Tile tables of the size classes for their own tile shapes: each class's domains (copies of
// the context's, re-tiled) with tile numbers starting at 0 within the class.
static int build_class_tables(snap_ctx *ctx) {
  const int nc = (int)ctx->cls.size();
  ctx->cls_dom.clear();
  ctx->cls_prefix.clear();
  ctx->cls_off.assign(nc, 0);
  for (int c = 0; c < nc; ++c) {
    const int *tl = ctx->ks.var[ctx->cls_tv[c]].tile;
    ctx->cls_off[c] = (int)ctx->cls_dom.size();
    int t = 0;
    ctx->cls_prefix.push_back(0);
    for (int i : ctx->cls[c]) {
      DomDev D = ctx->dom[i];
      D.tx = (D.nx + tl[0] - 1) / tl[0];
      D.ty = (D.ny + tl[1] - 1) / tl[1];
      D.tz = (D.nz + tl[2] - 1) / tl[2];
      D.tile_begin = t;
      t += D.tx * D.ty * D.tz;
      ctx->cls_dom.push_back(D);
      ctx->cls_prefix.push_back(t);
    }
    ctx->cls_ntiles[c] = t;
  }
  if (!ctx->cls_doms_dev) {
    CK(cudaMalloc(&ctx->cls_doms_dev, sizeof(DomDev) * ctx->ndom));
    CK(cudaMalloc(&ctx->cls_prefix_dev, sizeof(int) * (ctx->ndom + nc)));
  }
  CK(cudaMemcpyAsync(ctx->cls_doms_dev, ctx->cls_dom.data(), sizeof(DomDev) * ctx->ndom,
                     cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->cls_prefix_dev, ctx->cls_prefix.data(), sizeof(int) * (ctx->ndom + nc),
                     cudaMemcpyHostToDevice, ctx->stream));
  if (ctx->cls_streams.empty()) {
    ctx->cls_streams.assign(nc, nullptr);
    ctx->ev_join.assign(nc, nullptr);
    for (int c = 0; c < nc; ++c) {
      CK(cudaStreamCreateWithFlags(&ctx->cls_streams[c], cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&ctx->ev_join[c], cudaEventDisableTiming));
    }
    CK(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return SNAP_OK;
}

// One stage of every domain in the three-launch mode: a single launch over the context's
// tile table, or, with per-class tile shapes, one launch per size class on the classes'
// streams, forked from and joined back into s (parallel branches of a captured graph). The
// autotuner's only_class launches that class alone on s.
static int launch_stage(snap_ctx *ctx, const StageArgs &base, int stage, cudaStream_t s) {
  StageArgs a = base;
  a.stage = stage;
  if (!ctx->per_class && ctx->only_class < 0) {
    CK(ctx->ks.var[ctx->tv].stage(a, ctx->grid, s));
    return SNAP_OK;
  }
  const int nc = (int)ctx->cls.size();
  auto args_c = [&](int c) {
    StageArgs b = a;
    b.doms = ctx->cls_doms_dev + ctx->cls_off[c];
    b.tile_domain = ctx->cls_prefix_dev + ctx->cls_off[c] + c;
    b.ndom = (int)ctx->cls[c].size();
    b.ntiles = ctx->cls_ntiles[c];
    return b;
  };
  if (ctx->only_class >= 0) {
    const int c = ctx->only_class;
    CK(ctx->ks.var[ctx->cls_tv[c]].stage(args_c(c), ctx->cls_ntiles[c], s));
    return SNAP_OK;
  }
  CK(cudaEventRecord(ctx->ev_fork, s));
  for (int c = 0; c < nc; ++c) {
    CK(cudaStreamWaitEvent(ctx->cls_streams[c], ctx->ev_fork, 0));
    CK(ctx->ks.var[ctx->cls_tv[c]].stage(args_c(c), ctx->cls_ntiles[c], ctx->cls_streams[c]));
    CK(cudaEventRecord(ctx->ev_join[c], ctx->cls_streams[c]));
  }
  for (int c = 0; c < nc; ++c) CK(cudaStreamWaitEvent(s, ctx->ev_join[c], 0));
  return SNAP_OK;
}

// Tile index along one axis of the cell a ghost at position p (outside [0, n)) copies:
// wrapped on a periodic axis, mirrored at a wall.
static int ghost_source(int p, int n, bool periodic) {
  if (periodic) return ((p % n) + n) % n;
  return p < 0 ? -1 - p : 2 * n - 1 - p;
}

// Whether the resident step can run the current tiling: every tile co-resident, and no slab
// boundary (its ghost cells come from another domain's tiles).
static bool resident_possible(snap_ctx *ctx, std::string *why) {
  for (int i = 0; i < ctx->ndom; ++i)
    if (ctx->dom[i].bc[0] == kBcHalo || ctx->dom[i].bc[1] == kBcHalo) {
      if (why) *why = "the resident step does not take slab boundaries (SNAP_HALO)";
      return false;
    }
  const int mrt = ctx->ks.var[ctx->tv].max_resident_tiles();
  if (mrt <= 0 || ctx->ntiles > mrt) {
    if (why) *why = "the resident step needs every tile co-resident (" + std::to_string(ctx->ntiles) +
                    " tiles, " + std::to_string(mrt) + " co-resident CTAs for this tile shape)";
    return false;
  }
  return true;
}

// Ghost-cell dependencies of every tile for the resident step: the tiles holding the cells
// its three ghost layers per side copy (the same tile rows and columns, shifted along one
// axis, with the wrap or mirror of the domain boundary), made symmetric -- a tile that reads
// another's cells is also waited on by it, so no tile overwrites its state of a previous
// stage while a neighbour may still read it -- and without the tile itself.
static int build_resident(snap_ctx *ctx) {
  std::string why;
  if (!resident_possible(ctx, &why)) return fail(ctx, SNAP_ENOTSUP, "snap_use_persistent: " + why);
  const int *tl = ctx->ks.var[ctx->tv].tile;
  const int nt = ctx->ntiles;
  std::vector<std::vector<int>> dep(nt);
  for (int i = 0; i < ctx->ndom; ++i) {
    const DomDev &D = ctx->dom[i];
    const int n[3] = {D.nx, D.ny, D.nz}, tc[3] = {D.tx, D.ty, D.tz};
    const bool per[3] = {D.bc[0] == kBcPeriodic, D.bc[2] == kBcPeriodic, false};
    for (int t = 0; t < tc[0] * tc[1] * tc[2]; ++t) {
      const int ti[3] = {t % tc[0], (t / tc[0]) % tc[1], t / (tc[0] * tc[1])};
      for (int d = 0; d < 3; ++d) {
        if (n[d] == 1) continue;
        const int c0 = ti[d] * tl[d], c1 = std::min(c0 + tl[d], n[d]);
        for (int r = 1; r <= 3; ++r)
          for (int p : {c0 - r, c1 - 1 + r}) {
            const int q = (p >= 0 && p < n[d]) ? p : ghost_source(p, n[d], per[d]);
            int tj[3] = {ti[0], ti[1], ti[2]};
            tj[d] = q / tl[d];
            const int u = D.tile_begin + (tj[2] * tc[1] + tj[1]) * tc[0] + tj[0];
            if (u != D.tile_begin + t) dep[D.tile_begin + t].push_back(u);
          }
      }
    }
  }
  for (int t = 0; t < nt; ++t)
    for (int u : std::vector<int>(dep[t])) dep[u].push_back(t);
  std::vector<int> begin(nt + 1, 0), list;
  for (int t = 0; t < nt; ++t) {
    std::sort(dep[t].begin(), dep[t].end());
    dep[t].erase(std::unique(dep[t].begin(), dep[t].end()), dep[t].end());
    list.insert(list.end(), dep[t].begin(), dep[t].end());
    begin[t + 1] = (int)list.size();
  }
  cudaFree(ctx->tile_flags);
  cudaFree(ctx->dep_begin);
  cudaFree(ctx->dep_list);
  ctx->tile_flags = nullptr;
  ctx->dep_begin = ctx->dep_list = nullptr;
  CK(cudaMalloc(&ctx->tile_flags, sizeof(unsigned int) * nt));
  CK(cudaMalloc(&ctx->dep_begin, sizeof(int) * (nt + 1)));
  CK(cudaMalloc(&ctx->dep_list, sizeof(int) * (list.size() + 1)));
  CK(cudaMemsetAsync(ctx->tile_flags, 0, sizeof(unsigned int) * nt, ctx->stream));
  CK(cudaMemsetAsync(ctx->res, 0, sizeof(ResidentSync), ctx->stream));
  CK(cudaMemcpyAsync(ctx->dep_begin, begin.data(), sizeof(int) * (nt + 1),
                     cudaMemcpyHostToDevice, ctx->stream));
  if (!list.empty())
    CK(cudaMemcpyAsync(ctx->dep_list, list.data(), sizeof(int) * list.size(),
                       cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->res_ready = 1;
  ctx->res_tv = ctx->tv;
  return SNAP_OK;
}

static int enqueue_stages(snap_ctx *ctx, cudaStream_t s) {
  const TileVariant &tv = ctx->ks.var[ctx->tv];
  if (ctx->persistent == 2) {
    if (!ctx->res_ready) {
      int rc = build_resident(ctx);
      if (rc) return rc;
    }
    StageArgs a = args_of(ctx, 0);
    CK(tv.resident(a, ctx->ntiles, s));
    return SNAP_OK;
  }
  if (ctx->persistent) {
    // a barrier wait that gave up in an earlier launch leaves its arrival count behind:
    // every launch starts from a cleared barrier (a memset node in the captured graph)
    CK(cudaMemsetAsync(ctx->gsync, 0, sizeof(GridSync), s));
    StageArgs a = args_of(ctx, 0);
    CK(tv.step(a, ctx->grid_persistent, s));
    return SNAP_OK;
  }
  const StageArgs a = args_of(ctx, 0);
  for (int st = 0; st < 3; ++st) {
    const int rc = launch_stage(ctx, a, st, s);
    if (rc) return rc;
  }
  return SNAP_OK;
}

extern "C" int snap_stage(snap_ctx *ctx, int stage, double dt_fixed) {
  if (!ctx) return fail(nullptr, SNAP_EINVAL, "snap_stage: NULL context");
  if (stage < 0 || stage > 2) return fail(ctx, SNAP_EINVAL, "snap_stage: stage must be 0, 1 or 2");
  int rc = halos_ready(ctx, "snap_stage");
  if (rc) return rc;
  rc = set_dt_fixed(ctx, dt_fixed);
  if (rc) return rc;
  return launch_stage(ctx, args_of(ctx, 0), stage, ctx->stream);
}

extern "C" int snap_step_async(snap_ctx *ctx, int nsteps, double dt_fixed) {
  if (!ctx) return fail(nullptr, SNAP_EINVAL, "snap_step_async: NULL context");
  if (nsteps < 0) return fail(ctx, SNAP_EINVAL, "snap_step_async: nsteps < 0");
  if (nsteps == 0) return SNAP_OK;
  int rc = halos_ready(ctx, "snap_step_async");
  if (rc) return rc;
  if (ctx->persistent == 2 && !ctx->res_ready && (rc = build_resident(ctx))) return rc;
  rc = set_dt_fixed(ctx, dt_fixed);
  if (rc) return rc;
  if (!ctx->use_graph) {
    for (int n = 0; n < nsteps; ++n) {
      rc = enqueue_stages(ctx, ctx->stream);
      if (rc) return rc;
    }
    return SNAP_OK;
  }
  if (!ctx->graph) {
    cudaGraph_t g = nullptr;
    cudaStream_t cap = nullptr;
    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      rc = enqueue_stages(ctx, cap);
      cudaError_t e2 = cudaStreamEndCapture(cap, &g);
      if (rc == SNAP_OK && e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess && rc == SNAP_OK) e = cudaGraphInstantiate(&ctx->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (rc) return rc;
    if (e != cudaSuccess) {
      ctx->graph = nullptr;
      return cuda_fail(ctx, e, "snap_step_async: graph capture");
    }
  }
  for (int n = 0; n < nsteps; ++n) CK(cudaGraphLaunch(ctx->graph, ctx->stream));
  return SNAP_OK;
}

// Where a caller's buffer is for the device: 1 device (or managed) memory, 2 page-locked host
// memory mapped into the device (*dev set to its device address), 0 pageable host memory.
static int buffer_kind(const void *p, void **dev) {
  cudaPointerAttributes a;
  int kind = 0;
  *dev = nullptr;
  if (cudaPointerGetAttributes(&a, p) == cudaSuccess) {
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
      kind = 1;
      *dev = const_cast<void *>(p);
    } else if (a.type == cudaMemoryTypeHost && a.devicePointer) {
      kind = 2;
      *dev = a.devicePointer;
    }
  }
  cudaGetLastError();
  return kind;
}

extern "C" int snap_step_io(snap_ctx *ctx, int domain, const void *Y_in, void *Y_out, int dtype,
                            int nsteps, double dt_fixed) {
  if (!ctx) return fail(nullptr, SNAP_EINVAL, "snap_step_io: NULL context");
  if (domain < 0 || domain >= ctx->ndom || nsteps < 1 || (dtype != SNAP_F64 && dtype != SNAP_F32))
    return fail(ctx, SNAP_EINVAL, "snap_step_io: bad domain, nsteps or dtype");
  int rc;
  if (Y_in) {
    void *d = nullptr;
    const int kind = buffer_kind(Y_in, &d);
    if ((rc = snap_set_state(ctx, domain, Y_in, dtype, kind == 1, nullptr))) return rc;
  }
  if ((rc = snap_step_async(ctx, nsteps, dt_fixed))) return rc;
  if (!Y_out) return SNAP_OK;
  void *dst = nullptr;
  const int kind = buffer_kind(Y_out, &dst);
  return snap_get_state(ctx, domain, Y_out, dtype, kind == 1, nullptr);
}

static int read_status(snap_ctx *ctx, unsigned int *flags_out, int *sweeps_out) {
  unsigned int flags = 0;
  int sweeps = 0;
  CK(cudaMemcpyAsync(&flags, ctx->flags_dev, sizeof flags, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&sweeps, ctx->sweeps_dev, sizeof sweeps, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (flags_out) *flags_out = flags;
  if (sweeps_out) *sweeps_out = sweeps;
  return SNAP_OK;
}

extern "C" int snap_budget_compute(snap_ctx *ctx, int domain, snap_budget *out) {
  if (!ctx) return fail(nullptr, SNAP_EINVAL, "snap_budget_compute: NULL context");
  if (domain < 0 || domain >= ctx->ndom || !out) return fail(ctx, SNAP_EINVAL, "snap_budget_compute: bad arguments");
  StageArgs a = args_of(ctx, 0);
  const int nb = budget_blocks(ctx->dom[domain].ncell);
  CK(ctx->ks.budget(a, domain, 0, ctx->budget_partials, nb, ctx->budget_out, ctx->stream));
  double host[SNAP_MAX_FIELDS + 1];
  CK(cudaMemcpyAsync(host, ctx->budget_out, sizeof(double) * (ctx->nv + 1), cudaMemcpyDeviceToHost, ctx->stream));
  double dt = 0.0;
  CK(cudaMemcpyAsync(&dt, ctx->dt_dev + ctx->grp[domain], sizeof dt, cudaMemcpyDeviceToHost, ctx->stream));
  unsigned int flags = 0;
  int sweeps = 0;
  int rc = read_status(ctx, &flags, &sweeps);
  if (rc) return rc;
  memset(out, 0, sizeof *out);
  out->nfields = ctx->nv;
  for (int v = 0; v < ctx->nv; ++v) out->total[v] = host[v];
  out->energy_with_potential = host[ctx->nv];
  out->dt_last = dt;
  out->flags = flags;
  out->satadj_max_sweeps = sweeps;
  return SNAP_OK;
}

extern "C" int snap_check(snap_ctx *ctx, unsigned int *flags) {
  if (!ctx) return fail(nullptr, SNAP_EINVAL, "snap_check: NULL context");
  unsigned int f = 0;
  int rc = read_status(ctx, &f, nullptr);
  if (rc) return rc;
  if (flags) *flags = f;
  if (f & kFlagTimeout) return fail(ctx, SNAP_ETIMEOUT, "a grid barrier of the persistent step kernel timed out");
  if (f & kFlagNonFinite) return fail(ctx, SNAP_ENONFINITE, "a step produced a non-finite value or non-positive density");
  if (f & kFlagNoConv) return fail(ctx, SNAP_ENOCONV, "saturation adjustment did not converge in some cell");
  return SNAP_OK;
}

extern "C" int snap_step(snap_ctx *ctx, int nsteps, double dt_fixed, double *dt_used,
                         snap_budget *out_budget) {
  if (!ctx) return fail(nullptr, SNAP_EINVAL, "snap_step: NULL context");
  CK(cudaMemsetAsync(ctx->flags_dev, 0, sizeof(unsigned int), ctx->stream));
  int rc = snap_step_async(ctx, nsteps, dt_fixed);
  if (rc) return rc;
  if (dt_used) {
    CK(cudaMemcpyAsync(dt_used, ctx->dt_dev, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  }
  if (out_budget) {
    rc = snap_budget_compute(ctx, 0, out_budget);
    if (rc) return rc;
  }
  return snap_check(ctx, nullptr);
}

extern "C" int snap_reset_flags(snap_ctx *ctx) {
  if (!ctx) return fail(nullptr, SNAP_EINVAL, "snap_reset_flags: NULL context");
  CK(cudaMemsetAsync(ctx->flags_dev, 0, sizeof(unsigned int), ctx->stream));
  CK(cudaMemsetAsync(ctx->sweeps_dev, 0, sizeof(int), ctx->stream));
  return SNAP_OK;
}

extern "C" int snap_compute_dt(snap_ctx *ctx, int domain, double *dt) {
  if (!ctx) return fail(nullptr, SNAP_EINVAL, "snap_compute_dt: NULL context");
  if (domain < 0 || domain >= ctx->ndom || !dt) return fail(ctx, SNAP_EINVAL, "snap_compute_dt: bad arguments");
  int rc = refresh_rate(ctx, domain, ctx->stream);
  if (rc) return rc;
  unsigned long long bits = 0;
  CK(cudaMemcpyAsync(&bits, ctx->rate_dev + ctx->grp[domain], sizeof bits, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  double r;
  memcpy(&r, &bits, sizeof r);
  *dt = ctx->dom[domain].cfl / r;
  return SNAP_OK;
}

extern "C" int snap_saturation_adjust(snap_ctx *ctx, int domain) {
  if (!ctx) return fail(nullptr, SNAP_EINVAL, "snap_saturation_adjust: NULL context");
  if (domain < 0 || domain >= ctx->ndom) return fail(ctx, SNAP_EINVAL, "snap_saturation_adjust: bad domain");
  if (ctx->nvap == 0 || ctx->ncond == 0) return fail(ctx, SNAP_EINVAL, "snap_saturation_adjust: dry context");
  StageArgs a = args_of(ctx, 0);
  CK(ctx->ks.satadj(a, domain, 0, ctx->stream));
  int rc = refresh_rate(ctx, domain, ctx->stream);
  if (rc) return rc;
  return snap_check(ctx, nullptr);
}

static size_t state_bytes_dom0(snap_ctx *ctx) {
  return (size_t)ctx->dom[0].ncell * ctx->nv * ctx->word;
}

// Transpose of the saturation adjustment at the stage output Yout, on lam in place.
static int satadj_adjoint(snap_ctx *ctx, const StageArgs &sa, const void *Yout, void *lam) {
  AdjArgs A;
  memset(&A, 0, sizeof A);
  A.doms = ctx->doms_dev;
  A.Ys = Yout;
  A.lam_s = lam;
  A.ph = ctx->ph;
  A.cf = sa.cf;
  A.cd = sa.cd;
  CK(ctx->adj.satadj(A, ctx->dom[0].ncell, ctx->stream));
  return SNAP_OK;
}

// One forward stage; dt > 0 is passed in the launch arguments (the recorded time step). With
// ys/yn/yo set, the stage reads and writes those states instead of the domain's buffers.
static int plain_stage(snap_ctx *ctx, const StageArgs &base, int stage, double dt,
                       const void *ys = nullptr, const void *yn = nullptr, void *yo = nullptr,
                       cudaStream_t st = nullptr) {
  StageArgs a = base;
  a.stage = stage;
  a.dt_override = dt;
  a.buf_s = ys;
  a.buf_n = yn;
  a.buf_o = yo;
  CK(ctx->ks.var[ctx->tv].stage(a, ctx->grid, st ? st : ctx->stream));
  return SNAP_OK;
}

extern "C" int snap_record(snap_ctx *ctx, int nsteps, int ckpt_every, double dt_fixed) {
  if (!ctx) return fail(nullptr, SNAP_EINVAL, "snap_record: NULL context");
  if (!ctx->has_adj)
    return fail(ctx, SNAP_ENOTSUP, "snap_record: the adjoint is built for one inviscid domain, dry or with one vapour (x-z), free-slip or periodic sides, no fixed bottom temperature");
  if (nsteps < 1 || ckpt_every < 0)
    return fail(ctx, SNAP_EINVAL, "snap_record: nsteps must be >= 1 and ckpt_every >= 0");
  const size_t sb = state_bytes_dom0(ctx);
  const bool store_all = ckpt_every == 0;
  // store_all: the final state only; else every ckpt_every-th state and the final one
  const int nck = store_all ? 1 : (nsteps + ckpt_every - 1) / ckpt_every + 1;
  const int nseg_states = store_all ? nsteps : ckpt_every;
  ctx->rec_steps = 0;
  cudaFree(ctx->ckpt);
  cudaFree(ctx->segbuf);
  ctx->ckpt = ctx->segbuf = nullptr;
  CK(cudaMalloc(&ctx->ckpt, sb * nck));
  // per step: the inputs of its three stages (Y^n and the results of stages 0 and 1); with
  // more than one segment, room for two segments, so that the adjoint recomputes the next
  // segment while it transposes the current one (one segment's room if two do not fit)
  ctx->nsegbuf = 1;
  if (!store_all && nsteps > ckpt_every) {
    if (cudaMalloc(&ctx->segbuf, sb * 3 * nseg_states * 2) == cudaSuccess)
      ctx->nsegbuf = 2;
    else
      cudaGetLastError();
  }
  if (!ctx->segbuf) CK(cudaMalloc(&ctx->segbuf, sb * 3 * nseg_states));
  cudaFree(ctx->dt_hist);
  ctx->dt_hist = nullptr;
  CK(cudaMalloc(&ctx->dt_hist, sizeof(double) * nsteps));
  if (!ctx->lam) CK(cudaMalloc(&ctx->lam, sb * 4));
  if (!ctx->gface) {
    const DomDev &D = ctx->dom[0];
    size_t off = 0;
    for (int d = 0; d < 3; ++d) {
      if (d == 1 && !ctx->three_d) continue;
      long long nf = (long long)(D.nx + (d == 0)) * (D.ny + (d == 1)) * (D.nz + (d == 2));
      ctx->gface_off[d] = off;
      // per face and stencil slot, the fields padded to a 16-byte vector
      const int w = 16 / ctx->word, nvp = (ctx->nv + w - 1) / w * w;
      off += (size_t)nf * nvp * 6 * ctx->word;
    }
    CK(cudaMalloc(&ctx->gface, off));
  }
  if (!ctx->adjw && !ctx->f32) {
    // primitives [nv][ncell], then per direction 12 nv values per window centre (the cells
    // -1 .. n_d along the direction)
    const DomDev &D = ctx->dom[0];
    size_t off = (size_t)D.ncell * ctx->nv * 8;
    for (int d = 0; d < 3; ++d) {
      ctx->adjw_off[d + 1] = off;
      if (d == 1 && !ctx->three_d) continue;
      const long long nc = (long long)(D.nx + 2 * (d == 0)) * (D.ny + 2 * (d == 1)) * (D.nz + 2 * (d == 2));
      off += (size_t)nc * 12 * ctx->nv * 8;
    }
    CK(cudaMalloc(&ctx->adjw, off));
  }
  ctx->rec_dt.assign(nsteps, 0.0);
  ctx->ckpt_every = ckpt_every;
  const int keep = ctx->use_graph;
  const StageArgs base = args_of(ctx, 0);
  if (store_all) {
    int rc = set_dt_fixed(ctx, dt_fixed);
    if (rc) return rc;
  }
  for (int n = 0; n < nsteps; ++n) {
    if (store_all) {
      // three launches per step writing straight into the record: the inputs of the stages
      // of step n are slots 3n, 3n+1, 3n+2; stage 2 writes the next step's slot (the
      // context's state after the last step)
      const DomDev &D = ctx->dom[0];
      char *slot = (char *)ctx->segbuf + sb * 3 * n;
      if (n == 0) CK(cudaMemcpyAsync(slot, D.buf[0], sb, cudaMemcpyDeviceToDevice, ctx->stream));
      void *next = n + 1 < nsteps ? (void *)(slot + 3 * sb) : D.buf[0];
      int rc = plain_stage(ctx, base, 0, -1.0, slot, slot, slot + sb);
      if (!rc) rc = plain_stage(ctx, base, 1, -1.0, slot + sb, slot, slot + 2 * sb);
      if (!rc) rc = plain_stage(ctx, base, 2, -1.0, slot + 2 * sb, slot, next);
      if (rc) return rc;
    } else {
      if (n % ckpt_every == 0)
        CK(cudaMemcpyAsync((char *)ctx->ckpt + sb * (n / ckpt_every), ctx->dom[0].buf[0], sb,
                           cudaMemcpyDeviceToDevice, ctx->stream));
      int rc = snap_step_async(ctx, 1, dt_fixed);
      if (rc) return rc;
    }
    // the step's dt stays on the device until the end: no host round trip per step
    CK(cudaMemcpyAsync(ctx->dt_hist + n, ctx->dt_dev, sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  }
  CK(cudaMemcpyAsync((char *)ctx->ckpt + sb * (nck - 1), ctx->dom[0].buf[0], sb,
                     cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->rec_dt.data(), ctx->dt_hist, sizeof(double) * nsteps,
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->use_graph = keep;
  ctx->rec_steps = nsteps;
  return snap_check(ctx, nullptr);
}

// Adjoint of one stage: lam_s = b lam_out + (dL/dY_s)^T (b dt lam_out), and the step's
// initial-state adjoint lam_n according to mode (see AdjArgs).
static int adjoint_stage(snap_ctx *ctx, const StageArgs &sa, const void *Ys, const void *lo,
                         void *ls, void *ln, double a, double b, double dt, int mode) {
  AdjArgs A;
  memset(&A, 0, sizeof A);
  A.doms = ctx->doms_dev;
  A.Ys = Ys;
  A.lam_out = lo;
  A.lam_s = ls;
  A.lam_n = ln;
  A.a = a;
  A.b = b;
  A.dt = dt;
  A.mode = mode;
  A.ph = ctx->ph;
  A.cf = sa.cf;
  A.cd = sa.cd;
  const DomDev &D = ctx->dom[0];
  A.nx = D.nx;
  A.ny = D.ny;
  A.nz = D.nz;
  if (ctx->adjw) {
    A.X = ctx->adjw;
    for (int d = 0; d < 3; ++d) A.W[d] = (char *)ctx->adjw + ctx->adjw_off[d + 1];
  }
  long long ntot = 0;
  for (int d = 0; d < 3; ++d) {
    A.G[d] = (char *)ctx->gface + ctx->gface_off[d];
    if (d == 1 && !ctx->three_d) continue;
    ntot += (long long)(D.nx + (d == 0)) * (D.ny + (d == 1)) * (D.nz + (d == 2));
  }
  CK(ctx->adj.face(A, ntot, ctx->stream));
  CK(ctx->adj.cell(A, D.ncell, ctx->stream));
  return SNAP_OK;
}


extern "C" int snap_step_adjoint(snap_ctx *ctx, int nsteps, const void *lambda_final,
                                 void *lambda_init, int dtype, void *stream) {
  if (!ctx) return fail(nullptr, SNAP_EINVAL, "snap_step_adjoint: NULL context");
  if (!ctx->has_adj)
    return fail(ctx, SNAP_ENOTSUP, "snap_step_adjoint: the adjoint is built for one inviscid domain, dry or with one vapour (x-z), free-slip or periodic sides, no fixed bottom temperature");
  if (!lambda_final || !lambda_init || (dtype != SNAP_F64 && dtype != SNAP_F32))
    return fail(ctx, SNAP_EINVAL, "snap_step_adjoint: bad pointers or dtype");
  if (ctx->rec_steps < 1 || nsteps != ctx->rec_steps)
    return fail(ctx, SNAP_EINVAL, "snap_step_adjoint: nsteps must equal the steps of the last snap_record");
  cudaStream_t user = stream ? (cudaStream_t)stream : ctx->stream;
  CK(cudaStreamSynchronize(user));
  const DomDev &D = ctx->dom[0];
  const size_t sb = state_bytes_dom0(ctx);
  const long long n = D.ncell * ctx->nv;
  char *LA = (char *)ctx->lam, *LB = LA + sb, *LC = LB + sb, *LN = LC + sb;
  const int in_f32 = dtype == SNAP_F32;
  const size_t iw = in_f32 ? 4 : 8;
  cudaPointerAttributes pa;
  const bool dev_in = cudaPointerGetAttributes(&pa, lambda_final) == cudaSuccess &&
                      (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  const void *src = lambda_final;
  if (!dev_in) {
    CK(cudaMemcpyAsync(ctx->staging, lambda_final, n * iw, cudaMemcpyHostToDevice, ctx->stream));
    src = ctx->staging;
  }
  // an adjoint vector has no reference offset: plain type conversion
  CK(launch_state_copy(src, in_f32, LA, ctx->f32, ctx->nv, D.ncell, (long long)D.nx * D.ny,
                       nullptr, 1, ctx->stream));
  const bool store_all = ctx->ckpt_every == 0;
  const int K = store_all ? nsteps : ctx->ckpt_every;
  const int nseg = (nsteps + K - 1) / K;
  const StageArgs base = args_of(ctx, 0);
  const bool sa = ctx->adj.satadj && ctx->ph.satadj;
  // With two segment buffers the forward recomputation of segment seg - 1 runs on a second
  // stream while segment seg is transposed: the stage kernel and the adjoint kernels share
  // no buffer but the checkpoints (read-only); events order each buffer's reuse.
  const bool overlap = !store_all && ctx->nsegbuf == 2 && nseg > 1;
  if (overlap && !ctx->rec_stream) {
    CK(cudaStreamCreateWithFlags(&ctx->rec_stream, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
      CK(cudaEventCreateWithFlags(&ctx->ev_rec[b], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&ctx->ev_free[b], cudaEventDisableTiming));
    }
  }
  const size_t segb = sb * 3 * K;
  auto segment_buffer = [&](int seg) {
    return (char *)ctx->segbuf + (overlap ? segb * (seg & 1) : 0);
  };
  // recompute segment seg forward from its checkpoint, keeping Y^n and both intermediate
  // stages of each step
  auto recompute = [&](int seg, cudaStream_t st) -> int {
    const int n0 = seg * K, n1 = (n0 + K < nsteps) ? n0 + K : nsteps;
    char *buf = segment_buffer(seg);
    CK(cudaMemcpyAsync(buf, (char *)ctx->ckpt + sb * seg, sb, cudaMemcpyDeviceToDevice, st));
    for (int s = n0; s < n1; ++s) {
      char *slot = buf + sb * 3 * (s - n0);
      const double dt = ctx->rec_dt[s];
      int r;
      if ((r = plain_stage(ctx, base, 0, dt, slot, slot, slot + sb, st))) return r;
      if ((r = plain_stage(ctx, base, 1, dt, slot + sb, slot, slot + 2 * sb, st))) return r;
      if (s < n1 - 1 && (r = plain_stage(ctx, base, 2, dt, slot + 2 * sb, slot, slot + 3 * sb, st)))
        return r;
    }
    return SNAP_OK;
  };
  int rc = SNAP_OK;
  if (overlap) {
    // the recomputation stream starts after the work queued so far (the adjoint's input)
    CK(cudaEventRecord(ctx->ev_free[1], ctx->stream));
    CK(cudaStreamWaitEvent(ctx->rec_stream, ctx->ev_free[1], 0));
    rc = recompute(nseg - 1, ctx->rec_stream);
    if (!rc) CK(cudaEventRecord(ctx->ev_rec[(nseg - 1) & 1], ctx->rec_stream));
  }
  for (int seg = nseg - 1; seg >= 0 && rc == SNAP_OK; --seg) {
    const int n0 = seg * K, n1 = (n0 + K < nsteps) ? n0 + K : nsteps;
    const int b = seg & 1;
    if (overlap) {
      if (seg > 0) {
        // segment seg - 1 goes to the other buffer once the transpose of segment seg + 1
        // (its last reader) has finished with it
        if (seg + 1 < nseg) CK(cudaStreamWaitEvent(ctx->rec_stream, ctx->ev_free[b ^ 1], 0));
        if ((rc = recompute(seg - 1, ctx->rec_stream))) break;
        CK(cudaEventRecord(ctx->ev_rec[b ^ 1], ctx->rec_stream));
      }
      CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_rec[b], 0));
    } else if (!store_all) {
      if ((rc = recompute(seg, ctx->stream))) break;
    }
    char *buf = store_all ? (char *)ctx->segbuf : segment_buffer(seg);
    for (int s = n1 - 1; s >= n0 && rc == SNAP_OK; --s) {
      const double dt = ctx->rec_dt[s];
      const char *slot = (const char *)buf + sb * 3 * (s - n0);
      // Sec. 4.3 in reverse: Y3 = Y/3 + 2/3 (Y2 + dt L(Y2)), Y2 = 3/4 Y + 1/4 (Y1 + dt L(Y1)),
      // Y1 = Y + dt L(Y); each stage ends with the saturation adjustment, whose transpose is
      // taken at the stage's output first. The output of stage 2 is the next step's state:
      // the next slot, else the next checkpoint (the final state after the last step).
      const char *out2 = s + 1 < n1 ? slot + 3 * sb
                                    : (const char *)ctx->ckpt + sb * (store_all ? 0 : seg + 1);
      if (sa && (rc = satadj_adjoint(ctx, base, out2, LA))) break;
      if ((rc = adjoint_stage(ctx, base, slot + 2 * sb, LA, LB, LN, 1.0 / 3.0, 2.0 / 3.0, dt, 2))) break;
      if (sa && (rc = satadj_adjoint(ctx, base, slot + 2 * sb, LB))) break;
      if ((rc = adjoint_stage(ctx, base, slot + sb, LB, LC, LN, 0.75, 0.25, dt, 1))) break;
      if (sa && (rc = satadj_adjoint(ctx, base, slot + sb, LC))) break;
      if ((rc = adjoint_stage(ctx, base, slot, LC, LA, LN, 0.0, 1.0, dt, 0))) break;
    }
    if (overlap && rc == SNAP_OK) CK(cudaEventRecord(ctx->ev_free[b], ctx->stream));
  }
  // the recomputation stream's work is all waited for by the adjoint stream (an error
  // return may leave some queued: wait for it before the buffers are reused)
  if (overlap && rc != SNAP_OK) cudaStreamSynchronize(ctx->rec_stream);
  if (rc == SNAP_OK) {
    void *dst = lambda_init;
    cudaPointerAttributes po;
    const bool dev_out = cudaPointerGetAttributes(&po, lambda_init) == cudaSuccess &&
                         (po.type == cudaMemoryTypeDevice || po.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (!dev_out) dst = ctx->staging;
    CK(launch_state_copy(LA, ctx->f32, dst, in_f32, ctx->nv, D.ncell, (long long)D.nx * D.ny,
                         nullptr, 0, ctx->stream));
    if (!dev_out) CK(cudaMemcpyAsync(lambda_init, ctx->staging, n * iw, cudaMemcpyDeviceToHost, ctx->stream));
  }
  // restore the recorded final state
  const int nck = store_all ? 1 : (ctx->rec_steps + K - 1) / K + 1;
  CK(cudaMemcpyAsync(D.buf[0], (char *)ctx->ckpt + sb * (nck - 1), sb, cudaMemcpyDeviceToDevice, ctx->stream));
  int rc2 = refresh_rate(ctx, 0, ctx->stream);
  if (!rc) rc = rc2;
  CK(cudaStreamSynchronize(ctx->stream));
  return rc;
}

extern "C" int snap_theta_e(snap_ctx *ctx, int domain, double *out, int on_device) {
  if (!ctx) return fail(nullptr, SNAP_EINVAL, "snap_theta_e: NULL context");
  if (domain < 0 || domain >= ctx->ndom || !out) return fail(ctx, SNAP_EINVAL, "snap_theta_e: bad arguments");
  if (ctx->nvap != 1 || ctx->ncond < 1)
    return fail(ctx, SNAP_ENOTSUP, "snap_theta_e: defined for one vapour with a cloud");
  const DomDev &D = ctx->dom[domain];
  double *dst = out;
  if (!on_device) {
    CK(cudaMalloc(&dst, sizeof(double) * D.ncell));
  }
  cudaError_t e = launch_theta_e(ctx->doms_dev, domain, D.ncell, ctx->ph, ctx->f32, ctx->nv,
                                 ctx->three_d ? 3 : 2, dst, ctx->stream);
  if (e == cudaSuccess && !on_device)
    e = cudaMemcpyAsync(out, dst, sizeof(double) * D.ncell, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (!on_device) cudaFree(dst);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "snap_theta_e");
  return SNAP_OK;
}

extern "C" int snap_set_stream(snap_ctx *ctx, void *stream) {
  if (!ctx) return fail(nullptr, SNAP_EINVAL, "snap_set_stream: NULL context");
  ctx->stream = (cudaStream_t)stream;  // NULL: the legacy default stream
  return SNAP_OK;
}

extern "C" int snap_set_tile_variant(snap_ctx *ctx, int variant) {
  if (!ctx) return fail(nullptr, SNAP_EINVAL, "snap_set_tile_variant: NULL context");
  if (variant < 0 || variant >= ctx->ks.nvariants)
    return fail(ctx, SNAP_EINVAL, "snap_set_tile_variant: no such variant");
  return apply_variant(ctx, variant);
}

extern "C" int snap_set_class_tile_variant(snap_ctx *ctx, int cls, int variant) {
  if (!ctx) return fail(nullptr, SNAP_EINVAL, "snap_set_class_tile_variant: NULL context");
  if (cls < 0 || cls >= (int)ctx->cls.size() || variant < 0 || variant >= ctx->ks.nvariants)
    return fail(ctx, SNAP_EINVAL, "snap_set_class_tile_variant: no such size class or variant");
  ctx->cls_tv[cls] = variant;
  ctx->per_class = 1;
  if (ctx->graph) {
    cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
  }
  return build_class_tables(ctx);
}

extern "C" int snap_get_class_info(const snap_ctx *ctx, int cls, int *n_domains, int *cells,
                                   int tile[3], int *variant) {
  if (!ctx || cls < 0 || cls >= (int)ctx->cls.size()) return SNAP_EINVAL;
  const int v = ctx->per_class ? ctx->cls_tv[cls] : ctx->tv;
  const DomDev &D = ctx->dom[ctx->cls[cls][0]];
  if (n_domains) *n_domains = (int)ctx->cls[cls].size();
  if (cells) *cells = D.nx * D.ny * D.nz;
  if (tile)
    for (int i = 0; i < 3; ++i) tile[i] = ctx->ks.var[v].tile[i];
  if (variant) *variant = v;
  return SNAP_OK;
}

extern "C" int snap_use_persistent(snap_ctx *ctx, int enable) {
  if (!ctx) return fail(nullptr, SNAP_EINVAL, "snap_use_persistent: NULL context");
  if (enable < 0 || enable > 2) return fail(ctx, SNAP_EINVAL, "snap_use_persistent: mode 0, 1 or 2");
  if (enable == 1 && ctx->grid_persistent <= 0)
    return fail(ctx, SNAP_ECUDA, "snap_use_persistent: no co-resident CTA for the step kernel");
  if (enable == 2) {
    const int rc = build_resident(ctx);
    if (rc) return rc;
  }
  ctx->persistent = enable;
  if (ctx->graph) {
    cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
  }
  return SNAP_OK;
}

// Times `steps` steps of every tile variant in both launch modes on a copy of the current
// state, restores the state, and keeps the fastest. best_ms (may be NULL) gets its time per
// step; choice (may be NULL) gets variant * 2 + persistent.
extern "C" int snap_autotune(snap_ctx *ctx, int steps, double *best_ms, int *choice) {
  if (!ctx) return fail(nullptr, SNAP_EINVAL, "snap_autotune: NULL context");
  if (steps < 1) return fail(ctx, SNAP_EINVAL, "snap_autotune: steps < 1");
  // save every domain's state (and the CFL maxima) to restore after the trials
  size_t total = 0;
  for (int i = 0; i < ctx->ndom; ++i) total += (size_t)ctx->dom[i].ncell * ctx->nv * ctx->word;
  void *save = nullptr;
  CK(cudaMalloc(&save, total));
  std::vector<unsigned long long> rate(ctx->ndom);
  size_t off = 0;
  for (int i = 0; i < ctx->ndom; ++i) {
    size_t b = (size_t)ctx->dom[i].ncell * ctx->nv * ctx->word;
    CK(cudaMemcpyAsync((char *)save + off, ctx->dom[i].buf[0], b, cudaMemcpyDeviceToDevice, ctx->stream));
    off += b;
  }
  CK(cudaMemcpyAsync(rate.data(), ctx->rate_dev, sizeof(unsigned long long) * ctx->ndom,
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const int keep_graph = ctx->use_graph;
  ctx->use_graph = 0;
  double best = 1e300;
  int best_v = 0, best_p = 0, rc = SNAP_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (int v = 0; v < ctx->ks.nvariants && rc == SNAP_OK; ++v) {
    rc = apply_variant(ctx, v);
    for (int p = 0; p < 3 && rc == SNAP_OK; ++p) {
      if (p == 1 && ctx->grid_persistent <= 0) continue;
      if (p == 2 && !resident_possible(ctx, nullptr)) continue;
      ctx->persistent = p;
      rc = snap_step_async(ctx, 1, 0.0);  // warm-up
      if (rc) break;
      CK(cudaEventRecord(e0, ctx->stream));
      rc = snap_step_async(ctx, steps, 0.0);
      if (rc) break;
      CK(cudaEventRecord(e1, ctx->stream));
      CK(cudaEventSynchronize(e1));
      float ms = 0.0f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms / steps < best) {
        best = ms / steps;
        best_v = v;
        best_p = p;
      }
    }
  }
  // per size class: the fastest shape for each class launched alone, then the whole step with
  // every class on its own shape (three launches per class, in parallel) against the best
  // single shape
  const int nc = (int)ctx->cls.size();
  std::vector<int> cls_best(nc, 0);
  bool use_classes = false;
  auto time_steps = [&](double &ms_out) -> int {
    int r = snap_step_async(ctx, 1, 0.0);  // warm-up
    if (r) return r;
    CK(cudaEventRecord(e0, ctx->stream));
    r = snap_step_async(ctx, steps, 0.0);
    if (r) return r;
    CK(cudaEventRecord(e1, ctx->stream));
    CK(cudaEventSynchronize(e1));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    ms_out = ms / steps;
    return SNAP_OK;
  };
  if (nc > 1 && rc == SNAP_OK && ctx->ks.nvariants > 1) {
    ctx->persistent = 0;
    for (int c = 0; c < nc && rc == SNAP_OK; ++c) {
      double bc = 1e300;
      for (int v = 0; v < ctx->ks.nvariants && rc == SNAP_OK; ++v) {
        ctx->cls_tv[c] = v;
        ctx->only_class = c;
        if ((rc = build_class_tables(ctx))) break;
        double ms = 0.0;
        if ((rc = time_steps(ms))) break;
        if (ms < bc) {
          bc = ms;
          cls_best[c] = v;
        }
      }
    }
    ctx->only_class = -1;
    if (rc == SNAP_OK) {
      ctx->cls_tv = cls_best;
      ctx->per_class = 1;
      double ms = 0.0;
      if ((rc = build_class_tables(ctx)) == SNAP_OK && (rc = time_steps(ms)) == SNAP_OK &&
          ms < best) {
        best = ms;
        use_classes = true;
      }
      ctx->per_class = 0;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  off = 0;
  for (int i = 0; i < ctx->ndom; ++i) {
    size_t b = (size_t)ctx->dom[i].ncell * ctx->nv * ctx->word;
    CK(cudaMemcpyAsync(ctx->dom[i].buf[0], (char *)save + off, b, cudaMemcpyDeviceToDevice, ctx->stream));
    off += b;
  }
  CK(cudaMemcpyAsync(ctx->rate_dev, rate.data(), sizeof(unsigned long long) * ctx->ndom,
                     cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  cudaFree(save);
  ctx->use_graph = keep_graph;
  if (rc) return rc;
  rc = apply_variant(ctx, best_v);
  if (rc) return rc;
  ctx->persistent = best_p;
  if (use_classes) {
    ctx->persistent = 0;
    ctx->cls_tv = cls_best;
    ctx->per_class = 1;
    if ((rc = build_class_tables(ctx))) return rc;
  }
  if (best_ms) *best_ms = best;
  if (choice) *choice = use_classes ? -1 : best_v * 3 + best_p;
  CK(cudaMemsetAsync(ctx->flags_dev, 0, sizeof(unsigned int), ctx->stream));
  return SNAP_OK;
}

extern "C" int snap_set_barrier_test(snap_ctx *ctx, long long spin_cycles, int absent_cta) {
  if (!ctx) return fail(nullptr, SNAP_EINVAL, "snap_set_barrier_test: NULL context");
  if (spin_cycles < 0 || absent_cta < -1)
    return fail(ctx, SNAP_EINVAL, "snap_set_barrier_test: spin_cycles >= 0, absent_cta >= -1");
  ctx->spin_limit = spin_cycles > 0 ? spin_cycles : 4000000000ll;
  ctx->absent_cta = absent_cta;
  if (ctx->graph) {
    cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
  }
  return SNAP_OK;
}

extern "C" int snap_use_graph(snap_ctx *ctx, int enable) {
  if (!ctx) return fail(nullptr, SNAP_EINVAL, "snap_use_graph: NULL context");
  ctx->use_graph = enable ? 1 : 0;
  return SNAP_OK;
}

extern "C" int snap_get_info(const snap_ctx *ctx, snap_info *info) {
  if (!ctx || !info) return SNAP_EINVAL;
  info->n_domains = ctx->ndom;
  info->nfields = ctx->nv;
  info->ncells_total = ctx->ncells;
  info->state_bytes = ctx->state_bytes;
  for (int i = 0; i < 3; ++i) info->tile[i] = ctx->ks.var[ctx->tv].tile[i];
  info->tiles_total = ctx->ntiles;
  info->kernel_launches_per_step = ctx->persistent ? 1 : 3;
  info->tile_variant = ctx->tv;
  info->n_tile_variants = ctx->ks.nvariants;
  info->persistent = ctx->persistent;
  info->persistent_grid = ctx->grid_persistent;
  info->n_size_classes = (int)ctx->cls.size();
  info->per_class_tiles = ctx->per_class;
  if (ctx->per_class) info->kernel_launches_per_step = 3 * (int)ctx->cls.size();
  return SNAP_OK;
}

extern "C" int snap_link_halo(snap_ctx *ctx, int domain, int side, int nbr) {
  if (!ctx) return fail(nullptr, SNAP_EINVAL, "snap_link_halo: NULL context");
  if (domain < 0 || domain >= ctx->ndom || nbr < 0 || nbr >= ctx->ndom || (side != 0 && side != 1))
    return fail(ctx, SNAP_EINVAL, "snap_link_halo: bad domain, neighbour or side");
  DomDev &D = ctx->dom[domain];
  const DomDev &N = ctx->dom[nbr];
  if (D.bc[side] != kBcHalo || N.bc[1 - side] != kBcHalo)
    return fail(ctx, SNAP_EINVAL, "snap_link_halo: both facing sides must be SNAP_HALO");
  if (D.ny != N.ny || D.nz != N.nz || D.dz != N.dz || D.grav != N.grav ||
      ctx->rb_host[domain] != ctx->rb_host[nbr] || ctx->pf_host[domain] != ctx->pf_host[nbr])
    return fail(ctx, SNAP_EINVAL, "snap_link_halo: slabs of one domain need the same ny, nz, dz, "
                                  "grav and reference profile");
  for (int st = 0; st < 3; ++st) D.hsrc[side][st] = N.buf[st];
  D.hnx[side] = N.nx;
  D.hoff[side] = side == 0 ? N.nx - 3 : 0;
  ctx->halo_state[2 * domain + side] = 1;
  // one group, one CFL time step: the group of the lower index absorbs the other
  const int ga = ctx->grp[domain], gb = ctx->grp[nbr];
  const int keep = ga < gb ? ga : gb, drop = ga < gb ? gb : ga;
  for (int i = 0; i < ctx->ndom; ++i) {
    if (ctx->grp[i] == drop) ctx->grp[i] = keep;
    ctx->dom[i].rate = ctx->rate_dev + ctx->grp[i];
    ctx->dom[i].dt_step = ctx->dt_dev + ctx->grp[i];
  }
  CK(cudaMemcpyAsync(ctx->doms_dev, ctx->dom.data(), sizeof(DomDev) * ctx->ndom,
                     cudaMemcpyHostToDevice, ctx->stream));
  if (ctx->graph) {
    cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
  }
  if (ctx->per_class) {
    const int rc = build_class_tables(ctx);
    if (rc) return rc;
  }
  return refresh_rate(ctx, domain, ctx->stream);
}

extern "C" int snap_halo_buffer(snap_ctx *ctx, int domain, int side, void **ptr) {
  if (!ctx) return fail(nullptr, SNAP_EINVAL, "snap_halo_buffer: NULL context");
  if (domain < 0 || domain >= ctx->ndom || (side != 0 && side != 1) || !ptr)
    return fail(ctx, SNAP_EINVAL, "snap_halo_buffer: bad domain, side or pointer");
  if (ctx->dom[domain].bc[side] != kBcHalo || ctx->halo_state[2 * domain + side] == 1)
    return fail(ctx, SNAP_EINVAL, "snap_halo_buffer: not an unlinked SNAP_HALO side");
  const void *p = ctx->dom[domain].hsrc[side][0];
  *ptr = const_cast<void *>(p);
  ctx->halo_state[2 * domain + side] = 2;
  return SNAP_OK;
}

extern "C" int snap_halo_pack(snap_ctx *ctx, int domain, int side, int slot, void *out,
                              void *stream) {
  if (!ctx) return fail(nullptr, SNAP_EINVAL, "snap_halo_pack: NULL context");
  if (domain < 0 || domain >= ctx->ndom || (side != 0 && side != 1) || slot < 0 || slot > 2 || !out)
    return fail(ctx, SNAP_EINVAL, "snap_halo_pack: bad domain, side, slot or pointer");
  const DomDev &D = ctx->dom[domain];
  const long long nrow = (long long)D.ny * D.nz;
  const int x0 = side == 0 ? 0 : D.nx - 3;
  const long long n = (long long)ctx->nv * nrow * 3;
  const int grid = int(n / 256 + 1 < 1216 ? n / 256 + 1 : 1216);
  cudaStream_t s = pick(ctx, stream);
  if (ctx->f32)
    halo_pack_kernel<unsigned int><<<grid, 256, 0, s>>>(
        (const unsigned int *)D.buf[slot], (unsigned int *)out, ctx->nv, D.nx, nrow, x0);
  else
    halo_pack_kernel<unsigned long long><<<grid, 256, 0, s>>>(
        (const unsigned long long *)D.buf[slot], (unsigned long long *)out, ctx->nv, D.nx,
        nrow, x0);
  CK(cudaGetLastError());
  return SNAP_OK;
}

extern "C" int snap_buffer_pointer(snap_ctx *ctx, int domain, int slot, void **ptr) {
  if (!ctx || !ptr || domain < 0 || domain >= ctx->ndom || slot < 0 || slot > 2)
    return SNAP_EINVAL;
  *ptr = ctx->dom[domain].buf[slot];
  return SNAP_OK;
}

extern "C" void snap_free(snap_ctx *ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  release(ctx);
  delete ctx;
}

extern "C" const char *snap_last_error(const snap_ctx *ctx) {
  return ctx ? ctx->err.c_str() : g_init_error.c_str();
}

extern "C" const char *snap_status_string(int status) {
  switch (status) {
    case SNAP_OK: return "ok";
    case SNAP_EINVAL: return "invalid argument";
    case SNAP_ENOMEM: return "out of memory";
    case SNAP_ECUDA: return "CUDA error";
    case SNAP_ENONFINITE: return "non-finite value or non-positive density";
    case SNAP_ENOCONV: return "saturation adjustment did not converge";
    case SNAP_ETIMEOUT: return "device wait timed out";
    case SNAP_ENOTSUP: return "not supported by this build";
    default: return "unknown status";
  }
}
