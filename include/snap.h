/* snap.h -- C ABI of the GB300 (sm_103a) library for one explicit finite-volume step of the
 * compressible Euler equations with total energy and moist tracers, after
 * C. Li and X. Chen, "Simulating Non-hydrostatic atmospheres on Planets (SNAP)",
 * ApJS 2019 (arXiv 1901.02955).
 *
 * Conventions shared by every entry point
 *  - Return value: SNAP_OK (0) or a negative snap_status. No C++ exception crosses the ABI.
 *    snap_last_error() gives a one-line description of the last failure on a context.
 *  - A context is not thread-safe; use one host thread per context at a time.
 *  - Work is ordered on the context's CUDA stream (snap_set_stream; default: a stream the
 *    library creates). Calls that return host data synchronise that stream.
 *  - State layout (App. B conserved vector): structure of arrays Y[field][k][j][i], i fastest,
 *    interior cells only, fields in the order
 *      rho_d, rho_i (n_vapor), rho_ij (n_vapor x n_cond, grouped by vapour: i=0 j=0.., i=1 ..),
 *      rho u, [rho v when ny > 1], rho w, rho e.
 *    ny == 1 selects the x-z plane (no rho v). Units SI.
 *  - The library copies every input it is given; the caller keeps ownership of its buffers.
 *  - Internally the energy field is stored as rho e - pbar_k/(gamma_d - 1), the departure from
 *    the hydrostatic reference level by level, so that FP32 storage resolves pressure
 *    perturbations; set/get convert, and budgets report the total energy.
 */
#ifndef SNAP_H
#define SNAP_H

#ifdef __cplusplus
extern "C" {
#endif

#define SNAP_MAX_VAPOR 4
#define SNAP_MAX_COND 2
#define SNAP_MAX_FIELDS 24

typedef enum snap_status {
  SNAP_OK = 0,
  SNAP_EINVAL = -1,     /* invalid argument or descriptor */
  SNAP_ENOMEM = -2,     /* device or host allocation failed */
  SNAP_ECUDA = -3,      /* a CUDA call failed (snap_last_error has the CUDA message) */
  SNAP_ENONFINITE = -4, /* a step produced a non-finite value or a non-positive density */
  SNAP_ENOCONV = -5,    /* saturation adjustment hit its sweep limit in some cell */
  SNAP_ETIMEOUT = -6,   /* a bounded device-side wait gave up */
  SNAP_ENOTSUP = -7     /* combination of options not built into this library */
} snap_status;

/* Boundary of one side of a domain. SNAP_REFLECT: free-slip wall (ghost cells mirror the
 * state with the normal velocity negated). SNAP_PERIODIC: wrap (both opposite sides).
 * SNAP_NOSLIP: no-slip wall (ghost cells mirror the state with every velocity component
 * negated; Sec. 6 puts one at the bottom of the Jovian simulation). SNAP_HALO (x sides only):
 * the domain is one slab of a larger domain split along x, and the side's three ghost columns
 * are the neighbouring slab's cells, exchanged before every Runge-Kutta stage (the domain
 * decomposition over which Athena++, the paper's framework, parallelises a grid; see
 * snap_link_halo, snap_halo_buffer and snap_halo_pack). */
enum { SNAP_REFLECT = 0, SNAP_PERIODIC = 1, SNAP_NOSLIP = 2, SNAP_HALO = 3 };
enum { SNAP_F64 = 0, SNAP_F32 = 1 };

/* One condensable vapour i and its condensates (i,j); j = 0 is the cloud that exchanges mass
 * with the vapour in the saturation adjustment (App. D), j = 1 (precipitation) is carried. */
typedef struct snap_species {
  double eps;                   /* m_i / m_d (App. A) */
  double sigma_v;               /* c_v,i / c_v,d */
  double T_ref;                 /* reference temperature T^r of Eq. latent, K */
  double p_ref;                 /* saturation vapour pressure over condensate (i,0) at T_ref, Pa */
  double sigma_c[SNAP_MAX_COND];/* c_ij / c_v,d */
  double L_ref[SNAP_MAX_COND];  /* latent heat L^r_ij at T_ref, J/kg */
} snap_species;

/* Grid and physics of one domain (Sec. 2 equations, Sec. 4 scheme). */
typedef struct snap_grid_desc {
  int nx, ny, nz;          /* cells; ny == 1: x-z plane. Each active extent >= 3 */
  double dx, dy, dz;       /* cell sizes, m (dy ignored when ny == 1) */
  int bc[6];               /* x-, x+, y-, y+, z-, z+ : SNAP_REFLECT, SNAP_PERIODIC or
                              SNAP_NOSLIP, or SNAP_HALO on an x side; z must be walls; a
                              periodic side needs its opposite side periodic */
  double grav;             /* gravitational acceleration, m/s^2 (along -z) */
  double gamma_d;          /* c_p,d / c_v,d of the dry gas */
  double R_d;              /* dry-gas constant, J/(kg K) */
  int n_vapor;             /* 0 .. SNAP_MAX_VAPOR (library builds: 0, 1, 2) */
  int n_cond;              /* condensates per vapour: 0 or 2 */
  snap_species species[SNAP_MAX_VAPOR];
  const double *rho_bar;   /* host [nz]: reference density of each level */
  const double *p_bar_face;/* host [nz+1]: reference pressure at level faces, discretely
                              hydrostatic: p_face[k+1] = p_face[k] - grav rho_bar[k] dz
                              (checked to 1e-9 relative) */
  int dtype;               /* SNAP_F64 or SNAP_F32: storage and arithmetic of the step */
  double cfl;              /* dt = cfl / max_cells sum_d (|u_d| + c)/dx_d when no fixed dt */
  double nu;               /* constant kinematic viscosity, m^2/s (0: none; dry only) */
  int satadj;              /* 1: saturation adjustment after every stage (needs n_cond > 0) */
  int satadj_max_iter;     /* sweep limit of the adjustment (e.g. 20) */
  double satadj_tol;       /* relative stop tolerance on the molar transfer; raised to
                              32 machine epsilons of dtype when smaller, and for each vapour
                              to 4 (|a| + 2) epsilons, a the exponent of its saturation
                              pressure (the precision dtype holds that pressure to) */
  double weno_eps;         /* epsilon of the WENO5 weights (e.g. 1e-6) */
  /* Sec. 2, Eq. d3: terminal velocity of condensate j of every vapour, m/s (< 0 falls); a
   * nonzero value adds the sedimentation fluxes of mass, momentum and energy at z faces,
   * taken from the side the condensate comes from; nothing crosses the walls. Needs
   * n_cond > 0. */
  double w_term[SNAP_MAX_COND];
  /* Sec. 3: 1 applies the Kessler scheme after every step by backward Euler (needs n_cond ==
   * 2: condensate 0 cloud, 1 precipitation): kessler_k = k1 condensation, k2 autoconversion,
   * k3 accretion, k4 evaporation, 1/s; iterations stop at kessler_tol (raised as satadj_tol
   * is) or report SNAP_ENOCONV after kessler_max_iter. */
  int kessler;
  double kessler_k[4];
  int kessler_max_iter;
  double kessler_tol;
  /* Sec. 6 forcing of the Jovian simulation, by the reference pressure p_k of each level
   * (0 disables each): a body cooling of cool_rate K/s at constant volume (rho e loses C_v
   * cool_rate, C_v the mixture's heat capacity) where cool_p_lo <= p_k <= cool_p_hi; a sponge
   * relaxing the horizontal momenta at 1/(sponge_tau0 (p_k/sponge_p0)^2) where p_k <
   * sponge_p0, leaving rho e unchanged. Needs n_vapor > 0 (the library builds the forcing
   * into its moist kernels). */
  double cool_rate, cool_p_lo, cool_p_hi;
  double sponge_tau0, sponge_p0;
  /* Sec. 6 lower boundary (fixed temperature): > 0 holds the ghost cells below the bottom
   * wall at T_bottom (K). They keep the mirrored pressure, composition and velocities, so
   * their densities are the mirrored ones times T / T_bottom. Nothing is advected through
   * the wall (u* = 0 there); inviscid, the ghosts only enter the reconstruction next to the
   * wall; with viscosity the wall face carries the heat flux -rho c_p nu dT/dz. 0: off. */
  double T_bottom;
} snap_grid_desc;

/* Domain totals: field sums times the cell volume, and sum of (rho e + rho g z) dV. */
typedef struct snap_budget {
  int nfields;
  double total[SNAP_MAX_FIELDS];
  double energy_with_potential;
  double dt_last;          /* time step used by the last step, s */
  unsigned int flags;      /* bit 0: non-finite/non-positive density seen; bit 1: no conv. */
  int satadj_max_sweeps;   /* largest sweep count of the adjustment since the last reset */
} snap_budget;

typedef struct snap_ctx snap_ctx;

/* Create a context with n_domains >= 1 domains described by d[0..n_domains-1] (Sec. 2
 * equations on each). Domains of one context share dtype, n_vapor, n_cond, species table,
 * gamma_d, R_d, dimensionality and viscosity switch; sizes, spacings, boundaries, grav,
 * reference profiles and cfl may differ. n_domains > 1 advances all domains in the same
 * launches (an ensemble). Device memory: 3 state copies per domain plus small tables.
 * On success *out owns the context; release it with snap_free. */
int snap_init_grid(snap_ctx **out, const snap_grid_desc *d, int n_domains);

/* Copy the conserved state of one domain in. Y has the layout above with element type
 * dtype (SNAP_F64 or SNAP_F32, converted to the context's dtype); on_device != 0 means Y is a
 * device pointer (e.g. a torch CUDA tensor), else host memory: page-locked (pinned) memory
 * is read by the conversion kernel itself through its device mapping, asynchronously (keep
 * it unchanged until the stream has passed the call); pageable memory is staged. stream: a
 * cudaStream_t to order the copy on, or NULL for the context's. The CFL rate of the new
 * state is recomputed. */
int snap_set_state(snap_ctx *ctx, int domain, const void *Y, int dtype, int on_device,
                   void *stream);

/* Copy the current conserved state of one domain out (same layout and conventions). Host
 * destinations (pinned ones written directly by the conversion kernel) are complete when
 * the call returns. */
int snap_get_state(snap_ctx *ctx, int domain, void *Y_out, int dtype, int on_device,
                   void *stream);

/* Advance every domain by nsteps steps of SSP-RK3 (Sec. 4.3); each stage is the fused
 * WENO5 reconstruction (Sec. 4.2), LMARS flux (Sec. 4.1), flux divergence and gravity source
 * (Eq. forward), stage combine and saturation adjustment (App. D). dt_fixed > 0 uses that
 * time step for every domain; otherwise each domain uses its CFL rule from the state at the
 * start of each step. dt_used (may be NULL) receives domain 0's last time step; out_budget
 * (may be NULL) receives domain 0's budget after the last step. Returns SNAP_ENONFINITE or
 * SNAP_ENOCONV when a device check tripped during these steps (the state is still advanced). */
int snap_step(snap_ctx *ctx, int nsteps, double dt_fixed, double *dt_used,
              snap_budget *out_budget);

/* Enqueue nsteps steps on the context's stream and return at once: no host synchronisation,
 * no status read-back (use snap_check). Same dt_fixed meaning as snap_step. */
int snap_step_async(snap_ctx *ctx, int nsteps, double dt_fixed);

/* One call from a caller's state to the state nsteps steps later (Sec. 4.3 steps, as
 * snap_step_async), for one domain: snap_set_state, snap_step_async and snap_get_state with
 * the buffer kinds found by the library.
 *   Y_in   NULL (keep the context's state) or a state in the caller's layout of snap_set_state
 *          (device memory, page-locked or pageable host memory), read before the first step;
 *   Y_out  NULL or a buffer of the same layout for the state after the last step;
 *   dtype  SNAP_F32 or SNAP_F64, the type of Y_in and Y_out.
 * Returns when Y_out (if host memory) holds the result; with Y_out on the device or NULL the
 * work is only enqueued. No status read-back (use snap_check). SNAP_EINVAL for a bad domain,
 * nsteps < 1 or dtype; the errors of snap_set_state, snap_step_async and snap_get_state. */
int snap_step_io(snap_ctx *ctx, int domain, const void *Y_in, void *Y_out, int dtype, int nsteps,
                 double dt_fixed);

/* Enqueue one Runge-Kutta stage (0, 1 or 2 of Sec. 4.3) for every domain. Stage 0 reads the
 * state and writes the first intermediate, stage 1 the second, stage 2 writes the new state in
 * place; a step is the three in order. For timing and tests of single stages. */
int snap_stage(snap_ctx *ctx, int stage, double dt_fixed);

/* Synchronise the context's stream and report the device checks since the last reset:
 * SNAP_ENONFINITE, SNAP_ENOCONV or SNAP_OK; flags (may be NULL) receives the raw bits. */
int snap_check(snap_ctx *ctx, unsigned int *flags);

/* Clear the device check bits and the sweep-count maximum (stream-ordered). */
int snap_reset_flags(snap_ctx *ctx);

/* Budget of one domain's current state (FP64 sums, deterministic order). */
int snap_budget_compute(snap_ctx *ctx, int domain, snap_budget *out);

/* CFL time step of one domain's current state (what snap_step would use next). */
int snap_compute_dt(snap_ctx *ctx, int domain, double *dt);

/* Apply the App. D saturation adjustment to every cell of one domain's current state. */
int snap_saturation_adjust(snap_ctx *ctx, int domain);

/* Forward run recorded for the adjoint: advances the domain by nsteps steps like snap_step,
 * keeping the final state, the time step of every step and
 *   ckpt_every >= 1: a checkpoint of the state every ckpt_every steps; the adjoint recomputes
 *     each segment from its checkpoint. Allocates nsteps/ckpt_every + 2 state copies and a
 *     segment of 3 x ckpt_every states (the input of each of the three stages of a step);
 *   ckpt_every == 0: the input of every stage of every step (3 x nsteps + 1 state copies);
 *     the adjoint recomputes nothing.
 * Also allocates four adjoint vectors and the per-face work arrays of the adjoint. The
 * adjoint is built for a single inviscid domain, dry (x-z or 3-D) or with one vapour and two
 * condensates in the x-z plane, with free-slip or periodic sides and no fixed bottom
 * temperature; SNAP_ENOTSUP for any other context. */
int snap_record(snap_ctx *ctx, int nsteps, int ckpt_every, double dt_fixed);

/* Discrete adjoint of the recorded run: lambda_init = (dY_N / dY_0)^T lambda_final, with
 * Y_0 the state at the start of the last snap_record and Y_N the state at its end; nsteps
 * must equal the recorded step count. The transpose of each stage (saturation adjustment of
 * App. D, SSP-RK3 combine of Sec. 4.3, flux divergence and gravity source, LMARS of Sec.
 * 4.1, WENO5 of Sec. 4.2, primitive map of App. B) is applied in reverse order, segment by
 * segment, with the forward states of a segment recomputed from its checkpoint (or read from
 * the record when ckpt_every was 0). The recorded time steps are constants; the upwind side
 * of LMARS is held, except at u* = 0 where the mean of both one-sided derivatives is used;
 * the adjustment is differentiated through its equilibrium, with the set of vapours that
 * keep cloud held. Both vectors have the state layout (total energy; the reference offset
 * of the stored energy has unit derivative), dtype SNAP_F32/F64, host or device memory. The
 * context state is restored to Y_N afterwards. SNAP_ENOTSUP as for snap_record. */
int snap_step_adjoint(snap_ctx *ctx, int nsteps, const void *lambda_final, void *lambda_init,
                      int dtype, void *stream);

/* Equivalent potential temperature (App. A, Eq. theta_e) of every cell of one domain's
 * current state, for a context with one vapour whose first condensate is the cloud (q_t =
 * vapour + cloud; precipitation excluded), p0 = 1e5 Pa: theta_e = T (p0/p_d)^(R_d q_d / c)
 * exp(L q_v / (c T)), c = c_pd q_d + c_l q_t. out receives nx*ny*nz doubles in the state's
 * cell order, in device memory (on_device = 1) or host memory. Evaluated in FP64 whatever the
 * context's dtype. A diagnostic (the step does not use it); synchronous. SNAP_ENOTSUP for
 * other species tables. */
int snap_theta_e(snap_ctx *ctx, int domain, double *out, int on_device);

/* Order all following work of the context on this cudaStream_t. NULL selects the CUDA legacy
 * default stream (the handle of torch's default stream); a new context starts on a
 * non-blocking stream of its own. */
int snap_set_stream(snap_ctx *ctx, void *stream);

/* 1 (default): snap_step replays one captured CUDA graph per step; 0: plain launches. */
int snap_use_graph(snap_ctx *ctx, int enable);

/* Select one of the tile shapes built for the context's layout (count in
 * snap_info.n_tile_variants; the active one in snap_info.tile_variant). A new context starts
 * on the first shape, in the order built, whose tiles over all domains are at least the
 * device's SM count, else on the shape with the most tiles, so that a small grid still
 * spreads over every SM. Domains are re-tiled; results do not depend on the shape. */
int snap_set_tile_variant(snap_ctx *ctx, int variant);

/* Launch mode of a step. 0 (default): three launches per step, one per stage. 1: one
 * persistent cooperative launch whose CTAs (all co-resident) walk the tile queue of every
 * domain and meet at a grid barrier between the three stages. 2: the resident step, for grids
 * whose tiles are all co-resident at once (SNAP_ENOTSUP otherwise, or with SNAP_HALO sides):
 * one cooperative launch with one tile per CTA; each CTA keeps its tile's state on chip
 * through the three stages and, between stages, waits only for the tiles its ghost cells
 * come from (a flag per tile) instead of for the whole grid. Every device-side wait of modes
 * 1 and 2 is bounded (about 2 s) and reports SNAP_ETIMEOUT instead of hanging. Results are
 * the same in every mode. */
int snap_use_persistent(snap_ctx *ctx, int enable);

/* Test aid for the persistent step's grid barrier (the paper has no counterpart): each wait
 * spins at most spin_cycles SM clock cycles (0 restores the default, about 2 s) and CTA
 * absent_cta (-1: none) neither arrives at nor waits on the barriers, so that every other
 * CTA's wait runs out and the step reports SNAP_ETIMEOUT through snap_check / snap_step
 * instead of hanging. The results of such a step are not meaningful; every persistent
 * launch starts from a cleared barrier, so the next normal step is unaffected. Takes effect
 * from the next step (a captured graph is rebuilt). */
int snap_set_barrier_test(snap_ctx *ctx, long long spin_cycles, int absent_cta);
/* Autotuner: times `steps` steps of every tile shape in every launch mode that applies
 * (snap_use_persistent) on the current state, which is restored afterwards; with several
 * size classes it also times each class alone on every shape and then the step with every
 * class on its fastest shape, and keeps whichever configuration is fastest. best_ms (may be
 * NULL) receives its time per step; choice (may be NULL) variant * 3 + launch mode, or -1 for
 * per-class shapes (snap_get_class_info). Allocates one temporary copy of the state. */
int snap_autotune(snap_ctx *ctx, int steps, double *best_ms, int *choice);

/* Sizes the context was built with. */
typedef struct snap_info {
  int n_domains;
  int nfields;
  long long ncells_total;
  long long state_bytes;      /* bytes of one state copy over all domains */
  int tile[3];                /* cells per tile in x, y, z */
  int tiles_total;            /* tiles over all domains */
  int kernel_launches_per_step;
  int tile_variant;           /* active tile shape (see snap_set_tile_variant) */
  int n_tile_variants;
  int persistent;             /* 1: one cooperative launch per step */
  int persistent_grid;        /* CTAs of that launch (all co-resident) */
  int n_size_classes;         /* groups of domains of identical nx, ny, nz */
  int per_class_tiles;        /* 1: each size class on its own tile shape (see
                                 snap_set_class_tile_variant) */
} snap_info;
int snap_get_info(const snap_ctx *ctx, snap_info *info);
/* Tile shapes per size class. The domains of a context fall into size classes (identical
 * nx, ny, nz; numbered in the order of their first domain). snap_set_class_tile_variant
 * gives class cls its own tile shape (an index as for snap_set_tile_variant); from then on,
 * in the three-launch mode, every stage is one launch per class, the classes' launches
 * running in parallel on streams of the context (forked from and joined back into its
 * stream; parallel branches of the step's graph). snap_set_tile_variant returns every class
 * to the one shape. The persistent and resident modes run one kernel, so one shape: they
 * ignore the classes' shapes. snap_get_class_info reports a class's domain count, cells per
 * domain, tile shape and variant (NULL pointers are skipped). */
int snap_set_class_tile_variant(snap_ctx *ctx, int cls, int variant);
int snap_get_class_info(const snap_ctx *ctx, int cls, int *n_domains, int *cells, int tile[3],
                        int *variant);

/* Slab decomposition of one domain along x (the ghost cells of a SNAP_HALO side).
 *
 * snap_link_halo: within one context, the ghost columns of side `side` (0: x-, 1: x+) of
 * `domain` are read by the stage kernels straight from the stage input of domain `nbr` (its
 * last three columns for x-, its first three for x+): no copy, no extra launch. Both sides
 * must be SNAP_HALO (nbr's side 1 - side), and the two domains must have the same ny, nz, dz,
 * grav and reference profile. Linked domains form one group that shares a single CFL time
 * step (the largest rate over the group, as the undecomposed domain has), so a group
 * advances exactly like the whole domain: an x-periodic domain becomes a ring of slabs
 * (link the last slab's x+ to the first), a walled one a chain. Set up the links before
 * stepping; link each pair from both sides.
 *
 * snap_halo_buffer: for a neighbour in another context, process or GPU: *ptr receives the
 * device address of the side's ghost buffer, nfields x nz x ny x 3 values of the context's
 * dtype in the stored layout (i fastest; the energy field stored as rho e - pbar_k/(gamma_d
 * - 1), identical on both slabs of one domain), which the stage kernels read as the side's
 * ghost columns. The caller fills it before each stage with the neighbour's snap_halo_pack
 * output of the same stage input (e.g. an NCCL receive into it). Valid until snap_free.
 *
 * snap_halo_pack: writes the three columns of `domain` next to `side` of state buffer `slot`
 * (0, 1, 2: the input of stage 0, 1, 2; see snap_buffer_pointer) to the device buffer out in
 * the layout of snap_halo_buffer, ordered so that it is the opposite neighbour's ghost
 * buffer as it stands. Stream-ordered on stream (NULL: the context's).
 *
 * snap_step and snap_stage return SNAP_EINVAL while a SNAP_HALO side is neither linked nor
 * given to the caller through snap_halo_buffer. Contexts with SNAP_HALO sides have no
 * adjoint (SNAP_ENOTSUP). */
int snap_link_halo(snap_ctx *ctx, int domain, int side, int nbr);
int snap_halo_buffer(snap_ctx *ctx, int domain, int side, void **ptr);
int snap_halo_pack(snap_ctx *ctx, int domain, int side, int slot, void *out, void *stream);
/* Device pointer of one of a domain's three state buffers: slot 0 the current state, slot 1
 * the result of stage 0, slot 2 the result of stage 1 (dtype of the context, stored layout:
 * the energy field holds rho e - pbar_k/(gamma_d - 1)).
 * Valid until snap_free; the library writes them during stages. */
int snap_buffer_pointer(snap_ctx *ctx, int domain, int slot, void **ptr);

/* Budget of a state held in the caller's device memory, computed without any allocation by
 * the library. It serves callers that cannot allocate device memory and therefore cannot
 * create a context: code running under a fixed memory pool that must not grow, inside a
 * framework that owns all device memory and hands out only pre-sized tensors, or during a
 * phase in which cudaMalloc is not allowed. The paper has no counterpart; this is a service
 * of the library, a variant of the reduction behind snap_budget_compute.
 *   Y: device pointer in the caller's layout: nfields planes of nx*ny*nz values (i fastest),
 *      the first n_mass_fields planes densities, the last plane the total energy rho e;
 *      dtype SNAP_F32 or SNAP_F64.
 *   out: device pointer to nfields + 1 doubles: each field's sum times the cell volume, then
 *      the sum of (rho e + rho g z) times the cell volume (z at cell centres, dy ignored
 *      when ny == 1).
 *   stream: cudaStream_t to order the work on (NULL: the legacy default stream).
 * Scratch: a fixed device array of 1024 x 25 doubles (200 KiB) inside the library, held by
 * every device that loads the library until the process exits. nfields is limited to
 * SNAP_MAX_FIELDS (SNAP_EINVAL beyond). Each call writes every partial-sum row it later
 * reads, so nothing has to be cleared between calls; but all calls on a device share the
 * array, so calls whose work overlaps on the GPU (other streams, other host threads) race
 * and give wrong sums: serialise them. Every call made outside stream capture looks up the
 * array's device address in the device's current context (cudaGetSymbolAddress), so a
 * context destroyed and created again (cudaDeviceReset) is followed; a call on a capturing
 * stream reuses the address of the last call outside capture on that device, so make one
 * call before capturing (and again after a reset): with none, the call returns SNAP_ECUDA.
 * A CUDA error already pending in the process when the call starts is left in place for its
 * owner and reported as SNAP_ECUDA, with nothing launched.
 * Returns SNAP_OK, SNAP_EINVAL or SNAP_ECUDA; out is complete when the stream reaches it. */
int snap_budget_noalloc(const void *Y, int dtype, int nx, int ny, int nz, int nfields,
                        int n_mass_fields, double dx, double dy, double dz, double grav,
                        double *out, void *stream);

/* Arithmetic-throughput probe of the current device, a measurement aid (the paper has no
 * counterpart): chains of fused multiply-adds in the given type (SNAP_F32 or SNAP_F64) on
 * every SM, timed with CUDA events on stream (NULL: the legacy default stream) after warm-up
 * launches; *tflops receives the achieved rate at the clocks of the moment (2 flop per fused
 * multiply-add). Allocates nothing. Returns SNAP_OK, SNAP_EINVAL or SNAP_ECUDA. */
int snap_probe_fma(int dtype, double *tflops, void *stream);

/* Arithmetic self-checks, test aids that run pieces of the stage kernels on given arguments.
 * All pointers are device (or device-mapped) memory owned by the caller; the kernels run
 * asynchronously on stream. Allocate nothing. Return SNAP_OK, SNAP_EINVAL (a NULL pointer
 * with n > 0, n < 0, an unknown dtype, or a packed check that is not SNAP_F32 with n even)
 * or SNAP_ECUDA (launch failure).
 *
 * snap_check_rcp64: for the n doubles x, y[2i] = the FP64 kernels' reciprocal of x[i]
 * (Newton-Raphson from the approximate hardware reciprocal) and y[2i+1] = 1.0 / x[i] by IEEE
 * division.
 *
 * snap_check_weno: n windows of five values (a, b, c, d, e) = (Q_{c-2} .. Q_{c+2}) of the given
 * dtype, laid out [n][5]; out [n][2] receives the kernels' WENO5 states of Sec. 4.2 (Eq. weno5
 * with the Jiang-Shu indicators and the given eps): the left state at face c+1/2 and the
 * right state at face c-1/2. packed = 1 (SNAP_F32, n even) runs windows 2p and 2p+1 through
 * the packed two-variable form the FP32 kernels use for pairs of variables. */
int snap_check_rcp64(const double *x, double *y, long long n, void *stream);
int snap_check_weno(int dtype, int packed, const void *win, void *out, long long n, double eps,
                    void *stream);

void snap_free(snap_ctx *ctx);
const char *snap_last_error(const snap_ctx *ctx);
const char *snap_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif
