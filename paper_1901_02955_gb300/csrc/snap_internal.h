// snap_internal.h -- structures shared by the host library (capi.cu) and the kernel
// translation units. Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace snap {

constexpr int kMaxVap = 4;
constexpr int kMaxCond = 2;

// Physical constants of a context, derived on the host from snap_grid_desc (Sec. 2, App. A).
struct Phys {
  double gamma_d, R_d, c_vd, c_pd, kappa;  // kappa = R_d / c_pd
  int nvap, ncond;
  double eps[kMaxVap], inv_eps[kMaxVap];
  double sig_v[kMaxVap];                   // c_v,i / c_vd
  double sig_c[kMaxVap][kMaxCond];         // c_ij / c_vd
  double mu[kMaxVap][kMaxCond];            // chemical potential of condensate ij, mu_i = 0
  double Tref[kMaxVap], pref[kMaxVap];     // saturation curve over condensate (i,0)
  double beta[kMaxVap], delta[kMaxVap];    // Clausius-Clapeyron constants (App. D)
  double R_v[kMaxVap];                     // R_d / eps_i
  double sig_hat[kMaxVap];                 // molar c_v,i / c_vd = sigma_v,i * eps_i
  double weno_eps;
  double nu;
  int satadj, satadj_max_iter;
  double satadj_tol;
  double w_term[kMaxCond];                 // terminal velocity of condensate j (Eq. d3)
  int sediment;                            // any w_term != 0
  int kessler, kessler_max_iter;           // Kessler scheme (Sec. 3) after every step
  double kessler_k[4];                     // k1 .. k4
  double kessler_tol;
  double cool_rate, cool_p_lo, cool_p_hi;  // body cooling (Sec. 6), K/s in [p_lo, p_hi]
  double sponge_tau0, sponge_p0;           // sponge where p < p0 (Sec. 6)
};

// The same constants in the arithmetic type of a kernel, derived on the host, so that FP32
// kernels execute no double-precision conversion or arithmetic on their hot path.
template <class T>
struct CstT {
  T gamma_d, gm1, igm1, R_d, iR_d, kappa, c_pd, nu, weno_eps, satadj_tol;
  T eps[kMaxVap], inv_eps[kMaxVap], ieps_m1[kMaxVap], sig_v[kMaxVap], sigv_m1[kMaxVap];
  T sig_c[kMaxVap][kMaxCond], sigc_m1[kMaxVap][kMaxCond], mu[kMaxVap][kMaxCond];
  T pref[kMaxVap], beta[kMaxVap], delta[kMaxVap], inv_Tref[kMaxVap], sighat_m1[kMaxVap];
  T w_term[kMaxCond], kk[4], kessler_tol, c_vd;
  T cool_rate, cool_p_lo, cool_p_hi, sponge_itau0, sponge_ip0;
};

// One domain as the kernels see it (device memory).
// Side boundary kinds (the values of SNAP_REFLECT, SNAP_PERIODIC, SNAP_NOSLIP).
enum BcKind : int { kBcReflect = 0, kBcPeriodic = 1, kBcNoSlip = 2, kBcHalo = 3 };

struct DomDev {
  int nx, ny, nz;
  int tx, ty, tz;            // tiles per direction
  int tile_begin;            // first tile index of this domain in the launch
  int bc[6];
  double dx, dy, dz;
  double grav, cfl, dt_fixed;
  long long ncell;
  void *buf[3];              // B0 = state, B1 = stage 1 result, B2 = stage 2 result
  const double *rho_bar;     // [nz]
  const double *p_face;      // [nz+1]
  const double *p_cell;      // [nz]
  const double *e_ref;       // [nz]: the stored energy field is rho e - e_ref[k],
                             // e_ref[k] = pbar_k / (gamma_d - 1) (hydrostatic reference)
  // FP32 copies for the FP32 kernels (no FP64 instruction on their hot path)
  const float *rb_hi;        // [nz] rho_bar rounded to FP32
  const float *rb_lo;        // [nz] rho_bar - rb_hi, so (rho - rb_hi) - rb_lo is accurate
  const float *pc_f;         // [nz]
  const float *pf_f;         // [nz+1]
  const float *er_f;         // [nz]
  double idx, idy, idz;      // inverse cell sizes
  float fidx, fidy, fidz, fgrav;
  unsigned long long *rate;  // CFL rate max as double bits (non-negative doubles order as
                             // unsigned integers)
  unsigned long long *rate_next;  // resident step: the next step's rate while it accumulates
  double *dt_step;           // time step of the current step
  double T_bot;              // > 0: temperature of the ghost cells below the bottom wall
  // ghost columns of a kBcHalo x side h (0: x-, 1: x+) for the input of stage s: source
  // array hsrc[h][s] of rows of hnx[h] cells (fields [nv][nz][ny][hnx]); ghost column c
  // (0..2, left to right) is source column hoff[h] + c
  const void *hsrc[2][3];
  int hnx[2], hoff[2];
};

// State of the grid-wide barrier of the persistent step kernel (device memory).
struct GridSync {
  unsigned int count;
  unsigned int gen;
};

// Launch bookkeeping of the resident step kernel (device memory): CTAs finished in the
// current launch, and the launch count that numbers the tile flags' stage epochs.
struct ResidentSync {
  unsigned int done;
  unsigned int seq;
};

struct StageArgs {
  const DomDev *doms;        // device array
  const int *tile_domain;    // device array [ndom+1]: prefix of tiles per domain
  int ndom;
  int ntiles;
  int stage;                 // 0, 1, 2
  unsigned int *flags;       // bit 0 non-finite, bit 1 no convergence
  int *max_sweeps;
  GridSync *gsync;           // persistent step kernel only
  long long spin_limit;      // clock cycles a grid-barrier wait spins before giving up
  // resident step kernel only: launch bookkeeping, per-tile stage flags, and per tile the
  // tiles its ghost cells come from (dep_list[dep_begin[t] .. dep_begin[t+1]))
  ResidentSync *res;
  unsigned int *tile_flags;
  const int *dep_begin, *dep_list;
  int absent_cta;            // test aid: this CTA skips its barrier arrivals (-1: none)
  double dt_override;        // > 0: time step of this launch, before any domain setting
  // single-domain launches only: when set, the stage reads its input from buf_s and Y^n from
  // buf_n and writes its output to buf_o instead of the domain's buffers
  const void *buf_s, *buf_n;
  void *buf_o;
  Phys ph;
  CstT<float> cf;
  CstT<double> cd;
};

enum Flag : unsigned int { kFlagNonFinite = 1u, kFlagNoConv = 2u, kFlagTimeout = 4u };

// One tile shape of a kernel family.
struct TileVariant {
  int tile[3];
  int threads;
  size_t smem_stage;
  cudaError_t (*stage)(const StageArgs &, int grid, cudaStream_t);
  // all three stages in one cooperative launch with grid barriers in between
  cudaError_t (*step)(const StageArgs &, int grid, cudaStream_t);
  int (*max_resident_blocks)();  // co-resident CTAs of the step kernel on this device
  cudaError_t (*prepare)();      // one-time attribute setup (dynamic shared memory)
  // all three stages in one cooperative launch, one tile per CTA, neighbour flags between
  // stages (grid = number of tiles, at most max_resident_tiles())
  cudaError_t (*resident)(const StageArgs &, int grid, cudaStream_t);
  int (*max_resident_tiles)();
};

constexpr int kMaxVariants = 4;

// Kernel family entry points (one per instantiated layout and type).
// N consecutive values of type T moved as one aligned access (16 bytes for 4 floats).
template <class T, int N>
struct alignas(sizeof(T) * N) Pack {
  T x[N];
};

struct KernelSet {
  int nvariants;
  TileVariant var[kMaxVariants];
  cudaError_t (*rate)(const StageArgs &, int dom, int buf, cudaStream_t);
  // a caller-layout state (FP32 or FP64, device-accessible) into the domain's stored state,
  // with the CFL rate of the result folded into the domain's rate slot
  cudaError_t (*load)(const void *src, int src_f32, const StageArgs &, int dom, long long plane,
                      long long nz, cudaStream_t);
  cudaError_t (*budget)(const StageArgs &, int dom, int buf, double *partials, int nblocks,
                        double *out, cudaStream_t);
  cudaError_t (*satadj)(const StageArgs &, int dom, int buf, cudaStream_t);
};

// Arguments of the adjoint kernels of one stage (dry, inviscid, single domain).
struct AdjArgs {
  const DomDev *doms;
  const void *Ys;        // stage input state (context type, stored layout)
  const void *lam_out;   // adjoint of the stage output (context type, state layout)
  void *lam_s;           // adjoint of the stage input (written)
  void *lam_n;           // accumulator of the adjoint of the step's initial state
  double a, b, dt;       // stage output = a Y^n + b (Y_s + dt L(Y_s))
  int mode;              // 2: lam_n = a lam_out; 1: lam_n += a lam_out; 0: lam_s = lam_n + ...
  void *G[3];            // per-direction face contributions [nfaces_d][6][nv padded to 16 B]
  // FP64 adjoint only: primitives of every cell of Ys [nv][ncell], and per direction the face
  // states and WENO gradients of every window centre [12 nv][ncentres_d] (see adj_weno_kernel)
  void *X;
  void *W[3];
  int nx, ny, nz;        // domain size (host copy, for the launch shapes)
  Phys ph;
  CstT<float> cf;
  CstT<double> cd;
};

struct AdjKernels {
  // faces of every direction in one launch (nfaces: total over the directions)
  cudaError_t (*face)(const AdjArgs &, long long nfaces, cudaStream_t);
  cudaError_t (*cell)(const AdjArgs &, long long ncell, cudaStream_t);
  // transpose of the saturation adjustment at the stage output Ys, applied to lam_s in
  // place (nullptr for dry layouts)
  cudaError_t (*satadj)(const AdjArgs &, long long ncell, cudaStream_t);
};

// Equivalent potential temperature of one domain's state (diag.cu), FP64 into out[ncell].
cudaError_t launch_theta_e(const DomDev *doms_dev, int dm, long long ncell, const Phys &ph,
                           int f32, int nv, int nmom, double *out, cudaStream_t s);

// Adjoint kernels of the inviscid single-domain layouts; false when not built.
bool find_adjoint_kernels(int f32, int nvap, int ncond, int three_d, AdjKernels *out);

// Returns false when the configuration is not built into this library.
bool find_kernels(int f32, int nvap, int ncond, int three_d, int visc, int micro, KernelSet *out);

// Number of partial rows the budget kernel writes for a domain of ncell cells.
int budget_blocks(long long ncell);

// Copy a state between the caller's layout (total energy) and the stored one (energy minus
// e_ref per level), converting FP32/FP64. to_stored = 1: caller -> stored.
cudaError_t launch_state_copy(const void *src, int src_f32, void *dst, int dst_f32, int nv,
                              long long ncell, long long plane, const double *e_ref,
                              int to_stored, cudaStream_t s);

}  // namespace snap
