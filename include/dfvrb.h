/*
 * dfvrb.h -- C ABI of the GB300 (sm_103a) diffuse rigid-body finite-volume
 * library: the explicit Eulerian cell update of Wallis, Barton & Nikiforakis,
 * "A unified diffuse interface method for the interaction of rigid bodies with
 * elastoplastic solids and multi-phase mixtures" (arXiv:2111.11806).
 *
 * The calls follow the paper's statement of the problem (Sec. 3, eq:sys_vec_form):
 * a uniform Cartesian grid, materials, initial primitive fields including the
 * rigid field r, a time step from the CFL condition, then steps of seeding
 * (Sec. 3.2) and SSP-RK3 (Sec. 3.1).
 *
 * Conventions used by every call
 *  - Status: every call returns dfv_status, 0 on success, < 0 on error.  No
 *    C++ exception crosses the ABI.  dfv_last_error(grid) gives a message for
 *    the last error on that grid (a static or grid-owned string).
 *  - Memory: the library allocates NO device memory.  The caller provides one
 *    device workspace of at least dfv_workspace_bytes() bytes (256-byte
 *    aligned) and keeps it alive until dfv_destroy(); the library places all
 *    state planes, temporaries and reduction scratch in it.  Host buffers are
 *    owned by the caller and are only read or written during the call.
 *  - Streams: all device work of a grid is issued on the cudaStream_t passed
 *    at creation (NULL = legacy default stream).  Calls that return host data
 *    (dfv_compute_dt, dfv_get_fields to host, dfv_get_body, dfv_check)
 *    synchronise that stream.
 *  - Field layout: structure of arrays, one plane per variable, planes stored
 *    one after another, each plane ncell = n0*n1*n2 doubles with x fastest
 *    (cell (i,j,k) at i + n0*(j + n1*k)).
 *    Primitive planes (N materials, d dimensions, nv stretch components):
 *        phi_1..phi_{N-1}, rho_1..rho_N, u_1..u_d, p, V_1..V_nv, r [, eps_1..eps_N]
 *    Conserved planes, same count and order of groups:
 *        phi_1..phi_{N-1}, (phi rho)_1..(phi rho)_N, (rho u)_1..(rho u)_d, rho E, V_1..V_nv, r
 *        [, (phi rho eps)_1..(phi rho eps)_N]
 *    (the bracketed plastic-strain planes only with dfv_options.solid = 2)
 *    nv = 0 for fluids; for solids nv = 3 (1-D: xx,yy,zz) or 5 (2-D:
 *    xx,xy,yx,yy,zz).  With N = 1 there is no phi plane and the single
 *    density plane is rho.
 *  - Boundaries: bc[2*d] / bc[2*d+1] for the low / high side of direction d:
 *    DFV_BC_TRANSMISSIVE (zero-gradient halo), DFV_BC_REFLECTIVE (slip wall)
 *    or DFV_BC_PERIODIC (both sides of a direction must then be periodic).
 */
#ifndef DFVRB_H
#define DFVRB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int dfv_status;

#define DFV_OK 0
#define DFV_ERR_ARG (-1)          /* invalid argument or call order */
#define DFV_ERR_CUDA (-2)         /* a CUDA runtime call failed */
#define DFV_ERR_NONPHYSICAL (-3)  /* a kernel saw rho <= 0, c^2 <= 0 or NaN */
#define DFV_ERR_TIMEOUT (-4)      /* a host wait exceeded its time limit */
#define DFV_ERR_WORKSPACE (-5)    /* workspace too small or misaligned */
#define DFV_ERR_UNSUPPORTED (-6)  /* combination not built (3-D solids; 3-D FP64 with
                                     three materials, whose tile exceeds shared memory) */
#define DFV_ERR_TOO_LARGE (-7)    /* grid larger than a fixed-size scratch allows */

#define DFV_FP64 0       /* plain FP64 everywhere */
#define DFV_FP32 1       /* FP32 storage, reconstruction and fluxes; FP64 in
                            closures of cells with a volume fraction < 1e-6
                            and in the polar decomposition */

#define DFV_BC_TRANSMISSIVE 0
#define DFV_BC_PERIODIC 1
#define DFV_BC_REFLECTIVE 2   /* slip wall: the halo mirrors the interior with the
                                 normal velocity and the stretch components with
                                 exactly one normal index negated */

#define DFV_MAT_IDEAL 0       /* p = (gamma-1) rho e                  (Sec. 2.1.3) */
#define DFV_MAT_STIFFENED 1   /* p = (gamma-1) rho e - gamma p_inf (Mie-Grueneisen form) */
#define DFV_MAT_ROMENSKII 2   /* eq:Romenskii with shear energy G J^2/rho (Sec. 2.1.3) */

#define DFV_FIELDS_CONSERVED 0
#define DFV_FIELDS_PRIMITIVE 1

typedef struct {
    double gamma;    /* ideal / stiffened: adiabatic index */
    double pinf;     /* stiffened: p_inf (Pa) */
    double rho0;     /* reference density: Romenskii rho0; for every kind the
                        phasic density used where the material is absent from
                        a cell (volume fraction < 1e-6); 0 = none (gases) */
    double K0;       /* Romenskii: bulk-like modulus */
    double G0;       /* Romenskii: shear modulus at rho0 */
    double alpha;    /* Romenskii: cold-curve exponent */
    double beta;     /* Romenskii: shear-modulus exponent */
    double Gamma0;   /* Romenskii: Grueneisen coefficient */
    double sigma_y;  /* yield stress for perfect plasticity (0: fluid) */
    /* Johnson-Cook flow stress (the paper's Table 2 gives these for copper),
     * used instead of sigma_y when jc_c1 > 0 or jc_c2 > 0:
     *   sigma_Y = (c1 + c2 eps_p^n)(1 + c3 ln max(rate/1 s^-1, 1))(1 - T*^m),
     *   T* = clip((T - 298 K)/(T_melt - 298 K), 0, 1),
     * eps_p the material's equivalent plastic strain (its history plane with
     * dfv_options.solid = 2, else 0), T = 298 K + (p - p_ref)/(rho Gamma C_V)
     * and rate the plastic strain a return at the rate-free yield stress would
     * remove over the step, divided by dt.  Needs T_melt > 298 K, C_V > 0. */
    double jc_c1, jc_c2;   /* Pa */
    double jc_c3, jc_n, jc_m;
    double jc_tmelt;       /* K */
    double jc_cv;          /* J/(kg K) */
} dfv_material_params;

typedef struct {
    int nmat;            /* number of materials, 1 to 3 */
    int solid;           /* 1: carry the stretch tensor V (elastoplastic); 2: also one
                            equivalent-plastic-strain plane (phi rho eps)_l per
                            material after r (Sec. 2.1.1 history variables; the
                            primitive plane is eps_l); 0: fluids */
    int use_thinc;       /* 1: MUSCL-BVD-THINC on phi and r (Sec. 3.1); 0: MUSCL only */
    double thinc_beta;   /* THINC steepness (1.6) */
    int hllc_lm;         /* 1: HLLC-LM flux (the low-Mach HLLC variant the paper
                            names for its cylinder test): the acoustic dissipation
                            of the star regions scaled by sin(min(1, Ma/0.1) pi/2),
                            Ma the larger face-normal Mach number; 0: HLLC */
    int seed_variant;    /* rigid seeding (Sec. 3.2, step 5): 0 the reflected
                            state; 1 the right star state of the HLLC problem
                            along the body normal between the reflected (left)
                            and the interpolated (right) state, whose normal
                            velocity is the body's */
    int normal_method;   /* body normal (Sec. 3.3): 0 Youngs, -grad r/|grad r|;
                            1 ELVIRA from the 3x3 block of r (2-D grids only,
                            else DFV_ERR_UNSUPPORTED) */
    int probe_mode;      /* probe (Sec. 3.2, step 2): 0 stepped, 1.0 .. 4.0 dx_min
                            until the 2^dim enclosing cells have r < 0.5; 1 fixed
                            1.5 dx_min whatever their r (seeded from the
                            step-start state: one extra launch per step) */
    int general_stage;   /* 0: the SSP-RK3 stages of a 2-D FP32 grid of one ideal or
                            stiffened gas (no solid, no periodic side, no HLLC-LM,
                            a static body) run in the warp-marching gas kernel,
                            the others in the general stage kernel; 1: always
                            the general stage kernel.  The two agree to FP32
                            rounding. */
    int gas_rows;        /* rows per work item of the gas kernel (a strip of 28
                            columns marches through that many rows): 0 chooses
                            from the total cell count (4 to 32), else 1 to 4096;
                            results do not depend on it */
    int seed_stages;     /* 1: seed the stage inputs too (U1 before stage 2, U3
                            before stage 3; Sec. 3.2 seeds the step-start state
                            only, 0); single grids only (a batch returns
                            DFV_ERR_UNSUPPORTED) */
} dfv_options;

typedef struct dfv_grid dfv_grid;

/* Bytes of device workspace a grid needs (all precisions and options given
 * here).  dim in 1..3; n[d] >= 1 for d < dim. */
dfv_status dfv_workspace_bytes(int dim, const int n[3], int nmat, int solid, int precision, size_t *bytes);

/* Create a grid on [lo, hi] with n cells per direction (Sec. 3: uniform
 * Cartesian mesh; the paper's AMR hierarchy is not built).  workspace: device
 * pointer, 256-byte aligned, >= dfv_workspace_bytes() bytes, owned by the
 * caller.  stream: a cudaStream_t or NULL.  On success *out owns host memory
 * only, released by dfv_destroy. */
dfv_status dfv_create_grid(int dim, const int n[3], const double lo[3], const double hi[3], const int bc[6],
                           int precision, const dfv_options *opt, void *workspace, size_t workspace_bytes,
                           void *stream, dfv_grid **out);

/* Add material number *id_out (0, 1, ... in call order; exactly opt->nmat
 * materials before dfv_set_fields).  Closures: Sec. 2.1.2-2.1.3. */
dfv_status dfv_add_material(dfv_grid *g, int kind, const dfv_material_params *p, int *id_out);

/* Initial fields from FP64 primitive planes (layout above).  on_device = 1:
 * `prim` is a device pointer; 0: host pointer.  Conversion to conserved
 * variables uses the mixture rules of Sec. 2.2.  Device fields and host
 * fields in page-locked memory registered with CUDA (cudaHostAlloc,
 * cudaHostRegister) are converted in place by the device; other host memory
 * is first copied into the grid's staging buffer.  A host call returns when
 * the buffer may be reused.  The same holds for every field call below. */
dfv_status dfv_set_fields(dfv_grid *g, const double *prim, int on_device);

/* Copy the current fields out as FP64 planes (layout above): which =
 * DFV_FIELDS_CONSERVED, the vector U of the reduced system (Sec. 2.1.1,
 * eq:sys_vec_form, with r, Sec. 2.3), or DFV_FIELDS_PRIMITIVE, the variables
 * of the reconstruction (Sec. 3.1) from the mixture rules of Sec. 2.2.
 * on_device selects a device or host destination; a host copy synchronises. */
dfv_status dfv_get_fields(dfv_grid *g, double *out, int which, int on_device);

/* The same two calls for a caller's padded structure-of-arrays buffer: plane
 * v starts plane_pitch elements after plane v-1 (plane_pitch >= the cell
 * count; the padding is neither read nor written).  DFV_ERR_ARG when
 * plane_pitch is below the cell count. */
dfv_status dfv_set_fields_pitched(dfv_grid *g, const double *prim, long long plane_pitch, int on_device);

/* Restore a state saved with dfv_get_fields(DFV_FIELDS_CONSERVED) (FP64
 * conserved planes, layout above; host or device, caller-owned): checkpoint
 * and resume.  The planes are stored as they are (FP64) or narrowed (FP32,
 * the exact inverse of the widening of dfv_get_fields), so that with the body
 * state (dfv_get_body / dfv_set_body) a resumed run continues bit for bit.
 * The grid's time t starts again at 0.  Returns when the host buffer may be
 * reused. */
dfv_status dfv_set_state(dfv_grid *g, const double *cons, int on_device);
dfv_status dfv_get_fields_pitched(dfv_grid *g, double *out, long long plane_pitch, int which, int on_device);

/* Rigid-body velocity v_r (Sec. 2.3, eq:revo), position and mass.  dynamic =
 * 1: after every step v += dt F/m, x += dt v with F the pressure force sum
 * over grad r (not in the paper, which imposes v_r).  Only dim components of
 * v are used. */
dfv_status dfv_set_body(dfv_grid *g, const double v[3], const double x[3], double mass, int dynamic);

/* The rigid body (Sec. 2.3): the pressure force of the last step, the sum
 * of p grad(r) dV over the seeded state (the discrete form of the surface
 * integral of -p n; not in the paper, which imposes v_r), and the body's
 * velocity v_r and position.  Synchronises; DFV_ERR_NONPHYSICAL if a kernel
 * flagged a state. */
dfv_status dfv_get_body(dfv_grid *g, double force[3], double v[3], double x[3]);

/* dt = cfl / max_cells sum_d (|u_d| + c)/dx_d (also covering the body speed)
 * on the current fields (Sec. 3: a fraction of the largest stable step).
 * Synchronises the stream; returns DFV_ERR_NONPHYSICAL if a kernel flagged
 * a non-physical state. */
dfv_status dfv_compute_dt(dfv_grid *g, double cfl, double *dt_out);

/* One time step of size dt: rigid seeding (Sec. 3.2), three SSP-RK3 stages of
 * the spatial operator of eq:spat_op (Sec. 3.1) with the thermodynamic
 * variables of rigid cells (r > 0.5) carried unchanged, plastic relaxation
 * (solids), body update (dynamic body).  Asynchronous on the stream. */
dfv_status dfv_step(dfv_grid *g, double dt);

/* `steps` steps with dt computed on the device each step from `cfl`
 * (clipped to land on t_end when t_end > 0), all launches on the stream with
 * no host synchronisation; the sequence of one step is captured once into a
 * CUDA graph and replayed.  *t_out (optional) receives the simulated time
 * (synchronises).  For a static body with the stepped probe, the end-of-step
 * update of the control block (time, next dt, rigid box) of each step runs in
 * the seeding launch of the next step, and that of the last step when a later
 * call needs it (dfv_run with a new cfl / t_end or with t_out, dfv_step,
 * dfv_compute_dt, dfv_get_body, dfv_set_body, dfv_set_fields, dfv_check):
 * results are identical, a step is four launches instead of five. */
dfv_status dfv_run(dfv_grid *g, int steps, double cfl, double t_end, double *t_out);

/* Synchronise the stream (waiting at most timeout_ms, <= 0: no limit) and
 * report DFV_ERR_NONPHYSICAL / DFV_ERR_TIMEOUT. */
dfv_status dfv_check(dfv_grid *g, int timeout_ms);

/* Per-kernel device timing of steps, with CUDA events recorded on the grid's
 * stream around each launch.  enable = 1 clears the record and starts
 * recording; enable = 0 stops, synchronises the stream and returns in
 * ms_out[0..4] the summed device time of the seeding, stage-1, stage-2 and
 * stage-3 launches and of the finalize (about 0 when it runs in the next
 * step's seeding launch), and in *steps_out the number of recorded
 * steps (either output may be NULL).  While recording, dfv_run launches the
 * kernels of each step directly instead of replaying a graph. */
dfv_status dfv_profile(dfv_grid *g, int enable, double ms_out[5], long long *steps_out);

/* Number of kernel launches issued by the library on this grid so far. */
dfv_status dfv_launch_count(const dfv_grid *g, long long *count);

/* Where the conserved state lies inside the caller's workspace, for reading
 * it in place (checkpoints, in-situ analysis) without dfv_get_fields:
 * off[0], off[1], off[2] = byte offsets of the planes of U^n (the current
 * state) and of the SSP-RK3 stage buffers U1 and U3 (Sec. 3.1); *pitch =
 * elements from one plane to the next (>= the cell count; the elements from
 * the cell count to pitch-1 of every plane are never written); *nvar = planes
 * (layout above); *elem_bytes = 8 (FP64) or 4 (FP32).  U^n is complete only
 * after the stream has finished the last step (dfv_check).  Any output may be
 * NULL. */
dfv_status dfv_state_layout(const dfv_grid *g, size_t off[3], long long *pitch, int *nvar, int *elem_bytes);

/* Release the grid's host memory (the grid of the problem statement,
 * Sec. 3).  The workspace stays the caller's; work already issued on the
 * stream is not waited for, so synchronise the stream before freeing the
 * workspace. */
dfv_status dfv_destroy(dfv_grid *g);

/* ---------------------------------------------------------------- batches
 * Many independent 2-D fluid instances of different sizes (own grid, rigid
 * body velocity and time step) advanced together: each phase of a step
 * (seeding, the three RK stages) is one persistent launch over a work list of
 * (instance, tile) items, and a step is captured once into a CUDA graph.  Each
 * instance follows exactly the single-grid algorithm above with its own dt.
 * Materials are shared by all instances.  Field layout per instance as for a
 * grid (index i selects the instance). */
typedef struct {
    int n[3];           /* cells per direction (n[2] unused) */
    double lo[3], hi[3];
    int bc[6];
    double v_body[3];   /* rigid-body velocity (static bodies: 0) */
} dfv_instance_desc;

typedef struct dfv_batch dfv_batch;

/* Workspace bytes of a batch (dim must be 2; fluids only, opt->solid = 0). */
dfv_status dfv_batch_workspace_bytes(int dim, int count, const dfv_instance_desc *desc, int precision,
                                     const dfv_options *opt, size_t *bytes);
/* Create a batch of `count` instances in the caller's workspace (256-byte
 * aligned device memory of at least dfv_batch_workspace_bytes). */
dfv_status dfv_batch_create(int dim, int count, const dfv_instance_desc *desc, int precision,
                            const dfv_options *opt, void *workspace, size_t workspace_bytes, void *stream,
                            dfv_batch **out);
/* Add material number k (ideal or stiffened gas) to every instance. */
dfv_status dfv_batch_add_material(dfv_batch *b, int kind, const dfv_material_params *p);
/* Initial primitive fields of instance i (FP64 planes, host or device). */
dfv_status dfv_batch_set_fields(dfv_batch *b, int i, const double *prim, int on_device);
dfv_status dfv_batch_get_fields(dfv_batch *b, int i, double *out, int which, int on_device);
/* The same for every instance in one call (Sec. 4 setup of many independent
 * problems): prim[i] / out[i] (count pointers, caller-owned, host or device
 * as on_device says) hold instance i's nvar FP64 planes of n[0] n[1] values.
 * The copies and conversions of all instances are issued back to back on the
 * batch's stream and the call returns when they are done (host buffers may
 * then be reused); page-locked host buffers are converted in place, without
 * the staging copy, as for dfv_set_fields. DFV_ERR_ARG for a null pointer (nothing is copied) or,
 * when reading, an instance whose fields were never set. */
dfv_status dfv_batch_set_all_fields(dfv_batch *b, const double *const *prim, int on_device);
dfv_status dfv_batch_get_all_fields(dfv_batch *b, double *const *out, int which, int on_device);
/* `steps` steps of every instance, each with its own dt = cfl / (its CFL
 * bound), clipped to t_end when t_end > 0; no host synchronisation. */
dfv_status dfv_batch_run(dfv_batch *b, int steps, double cfl, double t_end);
/* Time trial steps of every (CTAs per SM, item schedule) candidate and keep
 * the fastest; the fields and times are restored afterwards.  choice_out (may
 * be NULL) receives {ctas_per_sm, schedule}: ctas_per_sm 0 launches one CTA per
 * work item, k > 0 a persistent grid of k CTAs per SM; schedule 0 instance
 * order with static round-robin assignment, 1 largest instances first,
 * static, 2 largest instances first from a dynamic queue. */
dfv_status dfv_batch_autotune(dfv_batch *b, int trial_steps, double cfl, int choice_out[2]);
/* Set the persistent grid (CTAs per SM, clipped to the occupancy limit) and
 * the schedule explicitly. */
dfv_status dfv_batch_set_schedule(dfv_batch *b, int ctas_per_sm, int schedule);
/* Simulated time and current dt of instance i (synchronises). */
dfv_status dfv_batch_get_time(dfv_batch *b, int i, double *t, double *dt);
/* Per-phase event timing of steps (seed, stage 1, 2, 3), like dfv_profile. */
dfv_status dfv_batch_profile(dfv_batch *b, int enable, double ms_out[4], long long *steps_out);
dfv_status dfv_batch_launch_count(const dfv_batch *b, long long *count);
dfv_status dfv_batch_destroy(dfv_batch *b);
const char *dfv_batch_last_error(const dfv_batch *b);

/* Largest grid (cells) that dfv_compute_dt_noalloc accepts. */
#define DFV_NOALLOC_MAX_CELLS (16LL * 1024 * 1024)

/* The CFL time step of a conserved state that the caller already holds on the
 * device, computed without allocating anything -- for callers that cannot
 * call cudaMalloc (for example a solver embedded in a host code that owns and
 * pools all device memory, or one that must not allocate while other work is
 * running).  The paper has no counterpart: it is a packaging of the CFL
 * reduction of dfv_compute_dt, returning the same dt for the same state.
 *   dim, n, lo, hi, precision, opt: as for dfv_create_grid (bc not needed);
 *   kinds[l], params[l]: the opt->nmat materials, as for dfv_add_material;
 *   cons: device pointer to the conserved planes (layout above) stored as
 *     doubles (DFV_FP64) or floats (DFV_FP32), plane_pitch elements apart
 *     (plane_pitch >= ncell);
 *   v_body: body velocity (the bound also covers it; NULL = at rest);
 *   dt_out: host pointer, receives cfl / max_cells sum_d (|u_d| + c)/dx_d.
 * Scratch: a fixed device array inside the library (DFV_NOALLOC_MAX_CELLS/256
 * block partials and a small control block), held by every device that loads
 * the library until the process exits; larger grids return
 * DFV_ERR_TOO_LARGE.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture.  All calls on a device share the array: calls whose work overlaps
 * on the GPU (other threads, other streams) race and must be serialised by the
 * caller.  The call synchronises `stream` (a cudaStream_t or NULL). */
dfv_status dfv_compute_dt_noalloc(int dim, const int n[3], const double lo[3], const double hi[3], int precision,
                                  const dfv_options *opt, const int kinds[], const dfv_material_params params[],
                                  const void *cons, long long plane_pitch, const double v_body[3], double cfl,
                                  void *stream, double *dt_out);

const char *dfv_last_error(const dfv_grid *g);

#ifdef __cplusplus
}
#endif

#endif /* DFVRB_H */
