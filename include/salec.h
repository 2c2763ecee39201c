/*
 * salec.h -- C ABI of the GB300 (sm_103a) SALEc-2D time-step library.
 *
 * The library advances a 2D axisymmetric Eulerian (SALE) impact simulation with
 * perfectly matched absorbing layers: the Lagrangian step (Eqs. 1-2 of the paper),
 * the PML auxiliary terms and damping (Sect. 3, Eqs. 15-26), the Eulerian donor-cell
 * remap (Eqs. 3-5) and the Courant time step (Sect. 6, Eq. 14).  Every step of the
 * cycle runs in CUDA kernels on one GPU; nothing falls back to the CPU.
 *
 * Conventions
 *  - Every call returns a salec_status; out-parameters are written only on SALEC_OK.
 *    salec_last_error() gives a one-line reason for the last failure of a context.
 *  - Call order: salec_create -> salec_set_material (each material) -> salec_add_layer /
 *    salec_place_projectile -> salec_finalize -> salec_step / read-outs.  A call out of
 *    order returns SALEC_EORDER.
 *  - Memory: the device state lives in ONE caller-owned device buffer (e.g. a torch
 *    uint8 tensor) of salec_state_bytes() bytes, 256-byte aligned; the library borrows it
 *    until salec_destroy and never allocates device memory of its own.  Host buffers
 *    passed to read-out calls are caller-owned and written synchronously.
 *  - Streams: every kernel and copy is issued on the stream given to salec_create
 *    (a cudaStream_t passed as void*, NULL = legacy default stream).  salec_step only
 *    enqueues; read-out calls synchronise that stream.
 *  - Fields are row-major [j][i] with j = 0 at the bottom: cell fields nz x nr, vertex
 *    fields (nz+1) x (nr+1).  SI units.
 *  - A context is not thread-safe; distinct contexts may be used from distinct threads.
 */
#ifndef SALEC_H
#define SALEC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct salec_ctx salec_ctx;

typedef enum {
    SALEC_OK = 0,
    SALEC_EINVAL = 1,      /* bad argument (size, index, parameter out of range) */
    SALEC_ENOMEM = 2,      /* the state buffer is too small or misaligned */
    SALEC_ECUDA = 3,       /* a CUDA call failed (message in salec_last_error) */
    SALEC_EORDER = 4,      /* call made before/after the stage it belongs to */
    SALEC_EUNSTABLE = 5,   /* the device status word reports a non-positive volume or
                              density, a NaN, dt below dt_min, or a copy of the tiles at
                              rest that did not complete (see salec_get_scalars) */
    SALEC_ETIMEOUT = 6     /* a bounded device wait ran out (the persistent batch's grid
                              barrier); the runs' states are partly advanced */
} salec_status;

/* Arithmetic of the step.  SALEC_FP64: every field and operation in FP64.
 * SALEC_FP32MIX: fields, stencils and material laws in FP32, while the specific internal
 * energy and its updates, the Courant reduction and the conservation sums are FP64
 * (the state buffer is about half the size). */
enum { SALEC_FP64 = 0, SALEC_FP32MIX = 1 };

enum { SALEC_EOS_TILLOTSON = 0, SALEC_EOS_IDEAL_GAS = 1 };
enum { SALEC_STRENGTH_NONE = 0, SALEC_STRENGTH_COLLINS = 1 };
enum { SALEC_TOP_OUTFLOW = 0, SALEC_TOP_WALL = 1 };
enum { SALEC_BOTTOM_NOSLIP = 0, SALEC_BOTTOM_FREESLIP = 1 };

/* Grid, boundary and numerical parameters (Table 2 of the paper names the grid and the
 * PML widths p_r, p_b; Sect. 4 the boundary conditions; Sect. 6 the Courant number). */
typedef struct salec_grid {
    int nr, nz;            /* cells in r and z (>= 1 each) */
    int nmat;              /* materials, 1..3 */
    double dx;             /* cell size, m */
    int pml_right;         /* right absorbing strip width, cells (0 = none, < nr) */
    int pml_bottom;        /* bottom absorbing strip width, cells (0 = none, < nz) */
    double pml_R;          /* theoretical reflection coefficient R of Eq. 26, 0 < R < 1 */
    double pml_c;          /* wave speed c of Eq. 26; <= 0: max sqrt(A/rho0) of the Tillotson materials */
    double pml_alpha;      /* relaxation rate of the PML auxiliaries in units of c / (strip width); 0: none */
    double gravity;        /* m/s^2, acting in -z */
    double cfl;            /* Courant number C0 of Eq. 14 */
    double dt_init;        /* "previous" dt that limits the growth of the first step */
    double dt_max;         /* upper bound of dt */
    double dt_growth;      /* dt_{n+1} <= dt_growth * dt_n */
    double dt_min;         /* a step with dt < dt_min sets the unstable status */
    double av_cq, av_cl;   /* artificial viscosity constants (quadratic, linear) */
    double f_min;          /* a material with a smaller volume fraction is removed */
    int bc_top;            /* SALEC_TOP_OUTFLOW or SALEC_TOP_WALL */
    int bc_bottom;         /* SALEC_BOTTOM_NOSLIP or SALEC_BOTTOM_FREESLIP */
} salec_grid;

/* One material: Tillotson (1962) or ideal-gas EoS; optional Collins et al. (2004)
 * strength with scalar damage (Sect. 1 and Table 1 of the paper).  The Tillotson form is
 * evaluated at no less than 1e-12 rho0, its dilute limit: below that density the sound
 * speed is the value there and the pressure is scaled by rho / (1e-12 rho0), i.e. it stays
 * a rho I; c^2 is floored at 0.01 A / rho0. */
typedef struct salec_material {
    int eos;                                        /* SALEC_EOS_* */
    double rho0;                                    /* reference density, kg/m^3 */
    double A, B, E0, a, b, alpha, beta, Eiv, Ecv;   /* Tillotson constants (Pa, J/kg) */
    double gamma;                                   /* ideal-gas ratio of specific heats */
    int strength;                                   /* SALEC_STRENGTH_* */
    double Yi0, mui, Yim, Yd0, mud, Ydm;            /* intact / damaged yield surfaces */
    double G;                                       /* shear modulus, Pa */
    double eps_fb, B_dam, p_bd;                     /* failure strain max(eps_fb, B_dam (p - p_bd)) */
    double p_t;                                     /* tensile limit of intact material, <= 0 */
} salec_material;

/* Field codes for salec_get_field / salec_set_field. */
enum {
    SALEC_F_VOLFRAC0 = 0, SALEC_F_VOLFRAC1 = 1, SALEC_F_VOLFRAC2 = 2,  /* f_m */
    SALEC_F_DENS0 = 3, SALEC_F_DENS1 = 4, SALEC_F_DENS2 = 5,           /* rho_m */
    SALEC_F_IE = 6, SALEC_F_SRR = 7, SALEC_F_SZZ = 8, SALEC_F_SRZ = 9, SALEC_F_DAMAGE = 10,
    SALEC_F_PMAX = 11,                 /* running max of (matter pressure - p0(row)) */
    SALEC_F_VR = 12, SALEC_F_VZ = 13,  /* vertex velocity */
    SALEC_F_PRESSURE = 14,             /* matter pressure sum f_m p_m / sum f_m (read only) */
    /* PML auxiliaries (zero outside their strip): cells */
    SALEC_F_PHI1_B = 20, SALEC_F_PHI3_B = 21, SALEC_F_PSI2_B = 22,
    SALEC_F_PHI1_R = 23, SALEC_F_PHI3_R = 24, SALEC_F_PSI2_R = 25,
    /* PML auxiliaries: vertices */
    SALEC_F_PHI2R_B = 30, SALEC_F_PHI2Z_B = 31, SALEC_F_PSI1R_B = 32, SALEC_F_PSI1Z_B = 33,
    SALEC_F_PHI2R_R = 34, SALEC_F_PHI2Z_R = 35, SALEC_F_PSI1R_R = 36, SALEC_F_PSI1Z_R = 37
};

/* Bytes of the device state buffer for this grid (persistent state, per-step scratch,
 * reduction partials and tables).  grid must pass the same checks as salec_create. */
salec_status salec_state_bytes(const salec_grid* grid, int precision, size_t* bytes);

/* Create a context over a caller-owned device buffer dev_state of `bytes` bytes
 * (>= salec_state_bytes, 256-byte aligned) on CUDA stream `stream`.  The buffer is
 * borrowed until salec_destroy.  *out receives the context. */
salec_status salec_create(const salec_grid* grid, int precision, void* dev_state, size_t bytes,
                          void* stream, salec_ctx** out);

/* Set material `id` (0..nmat-1).  Must precede salec_finalize. */
salec_status salec_set_material(salec_ctx* ctx, int id, const salec_material* mat);

/* Non-uniform cells: column widths dr[nr] and row heights dz[nz] (m, positive, host
 * arrays read during the call).  Without this call every cell is grid->dx square.  The
 * paper's grids (Table 2) have a high-resolution zone of equal cells and extension zones
 * whose cells grow by a constant factor (1.05) up to a maximum spacing; positions are the
 * running sums of the sizes from the axis and from the bottom.  Cell (i,j) has volume
 * r_c dr dz per radian, the viscosity and the Courant condition use its smaller side.
 * Must precede every salec_add_layer / salec_place_projectile (SALEC_EORDER otherwise);
 * SALEC_EINVAL for a non-positive or non-finite size.  salec_courant_dt_noalloc assumes
 * uniform cells of grid->dx. */
salec_status salec_set_spacing(salec_ctx* ctx, const double* dr, const double* dz);

/* Fill the rows between heights zlo < zhi (m; fractional rows allowed) with material
 * `mat` at density rho (rho <= 0: rho0, or discrete hydrostatic equilibrium when gravity
 * > 0 and the material is Tillotson with I0 = 0), specific internal energy I0 and
 * vertical velocity vz.  A hydrostatic layer fills whole rows (SALEC_EINVAL otherwise).
 * Hydrostatic layers stack: one whose top row lies right below a row filled by an earlier
 * hydrostatic layer starts from that row's pressure and density (its overburden), so a
 * layered target (sediment over crust over mantle, Sect. 4 of the paper) is added from
 * the top down. */
salec_status salec_add_layer(salec_ctx* ctx, int mat, double zlo, double zhi, double rho,
                             double I0, double vz);

/* Place a sphere of `radius` (m) centred on the axis at height zc, moving with vertical
 * velocity vz, density rho (<= 0: rho0) and energy I0.  Cell fractions are r-weighted
 * 16 x 16 sub-samples; the sphere displaces layer material. */
salec_status salec_place_projectile(salec_ctx* ctx, int mat, double radius, double zc,
                                    double vz, double rho, double I0);

/* Build the initial state on the host (fractions, densities, vertex velocities, PML
 * profiles of Eq. 26, reference rows) and copy it to the device. */
salec_status salec_finalize(salec_ctx* ctx);

/* Enqueue nsteps full cycles on the context's stream (no host synchronisation).  Whole
 * chunks of 16 steps go out as one CUDA-graph launch each (captured on first use and
 * again after the block shapes change; plain launches while per-kernel timing is on or
 * where capture is not possible); the results are those of plain launches. */
salec_status salec_step(salec_ctx* ctx, int nsteps);

/* How salec_step runs a cycle.
 *   SALEC_STEP_FUSED   the Courant kernel, then one kernel over tiles of cells that stages
 *                      each tile with a halo of three cells in shared memory and runs
 *                      every phase of the cycle (Fig. 1a: EoS and viscosity, corner forces
 *                      and v^L, energy / strength / volume partition, VOF remap, momentum
 *                      remap, heat) on it, then the Courant rates of the new state for the
 *                      next step.  The fields it rewrites are read from one copy and
 *                      written to a second one inside the state buffer; read-outs bring
 *                      the current copy back first.  It moves a quarter of the phase
 *                      form's DRAM bytes per cell but computes each tile's halo cells
 *                      again; a quiescent tile (matter at rest at zero pressure, whole
 *                      fractions, no deviatoric stress, no strip, no gravity), on which
 *                      every phase returns its input, only reads and writes its state.
 *                      A tile found quiescent in the step before, with its eight
 *                      neighbours, is at rest: it is copied without a halo (by a
 *                      streaming kernel before the tile kernel, or by a copy kernel
 *                      beside it: salec_set_rest_copy), and the other tiles are queued
 *                      for the tile kernel (one CTA per resident slot of the device).
 *                      Default when grid->gravity == 0.
 *   SALEC_STEP_PHASES  six kernels over the whole grid and the Courant kernel, in place
 *                      (block shapes from salec_set_block_shapes / salec_autotune).
 *                      Default under gravity, where no tile is quiescent and this form,
 *                      which computes no cell twice, issues fewer instructions.
 * Both forms compute the same cycle with the same arithmetic per cell and vertex;
 * salec_set_step_form returns SALEC_EINVAL for another value, SALEC_EORDER before
 * salec_finalize. */
enum { SALEC_STEP_PHASES = 0, SALEC_STEP_FUSED = 1 };
salec_status salec_set_step_form(salec_ctx* ctx, int form);
int salec_get_step_form(const salec_ctx* ctx);

/* Fused form, tiles at rest.  A tile is at rest when it and its eight neighbours passed
 * the tile kernel's quiescence test in the step before (or, for the first fused step
 * after set-up, a host write or other steps, when the Courant-rate pass over that state
 * found them quiescent with fields already in the form the quiescent path writes).
 *   mode 0  every tile goes through the tile kernel;
 *   mode 1  (default) a streaming kernel copies the tiles at rest and queues the others
 *           before the tile kernel starts;
 *   mode 2  a scan kernel queues the tiles, and a copy kernel of one warp per SM
 *           on a second stream of the context moves the tiles at rest with bulk tensor
 *           copies while the tile kernel runs on the same SMs.  Available in the FP64 form
 *           for a uniform grid of one hydrodynamic material with nr even, where a CTA of
 *           each kernel fit on one SM together; elsewhere mode 2 runs as mode 1.
 * The copy returns bit for bit what the tile kernel would, so the mode changes no result,
 * only the work done and its order.  SALEC_EINVAL for a null context or another mode. */
salec_status salec_set_rest_copy(salec_ctx* ctx, int mode);

/* Synchronise and read the scalars: out[0] t, out[1] dt of the last step, out[2] step
 * count, out[3] status bits (1 non-positive volume/density, 2 NaN, 4 dt < dt_min, 8 the
 * copy of the tiles at rest beside the tile kernel did not complete: a wait ran out),
 * out[4] mass out through the top, out[5] mass removed by clean-up, out[6] mass added by
 * the PML damping, out[7] z-momentum out through the top.  Returns SALEC_EUNSTABLE
 * (with out written) when status != 0. */
salec_status salec_get_scalars(salec_ctx* ctx, double out[8]);

/* Set the time and the previous dt (restart). */
salec_status salec_set_time(salec_ctx* ctx, double t, double dt_prev);

/* Copy a field into host_out (n = nr*nz for cell fields, (nr+1)*(nz+1) for vertex
 * fields), or overwrite a field from host_in (tests, fault injection). */
salec_status salec_get_field(salec_ctx* ctx, int field, double* host_out, size_t n);
salec_status salec_set_field(salec_ctx* ctx, int field, const double* host_in, size_t n);

/* Crater read-out (surface where sum_m f_m crosses 1/2, scanned from the top and
 * interpolated between cell centres): heights[nr] per column, depth on the axis below
 * z_surface, diameter (twice the first radius beyond the deepest column where the
 * surface regains z_surface), and depth_profile[npts] at r_k = (k + 1/2) r_extent / npts
 * with r_extent = (nr - pml_right) dx.  heights / depth_profile may be NULL. */
salec_status salec_crater_profile(salec_ctx* ctx, double z_surface, int npts,
                                  double* depth_profile, double* heights, double* depth,
                                  double* diameter);

/* Conservation sums per radian: out[0] mass, out[1] z-momentum, out[2] kinetic energy,
 * out[3] internal energy (block sums on the device, FP64). */
salec_status salec_conservation(salec_ctx* ctx, double out[4]);

/* Checkpoint: the persistent part of the device state (fields, PML auxiliaries, tables,
 * scalars) as an opaque byte image of salec_checkpoint_bytes() bytes. */
salec_status salec_checkpoint_bytes(salec_ctx* ctx, size_t* bytes);
salec_status salec_get_state(salec_ctx* ctx, void* host, size_t bytes);
salec_status salec_set_state(salec_ctx* ctx, const void* host, size_t bytes);

/* The caller wrote the first salec_checkpoint_bytes() bytes of the state buffer itself (a
 * device-to-device copy of an earlier image, say) instead of through salec_set_state: the
 * current fields are those at the start of the buffer, and the next fused step forms the
 * Courant maximum of that state again.  SALEC_EORDER before salec_finalize. */
salec_status salec_state_changed(salec_ctx* ctx);

/* Number of kernel launches one step issues (for launch accounting): in the phase form
 * the six phases and the one-thread Courant kernel between phases 0 and 1 (7); in the
 * fused form the Courant kernel, the rest-tile kernel and the tile kernel (3), or, with the
 * tiles at rest copied beside the tile kernel, the Courant, scan, copy and tile kernels
 * (4); a sequence of fused steps that follows set-up, a host write or other steps adds one
 * pass of Courant rates first. */
int salec_launches_per_step(const salec_ctx* ctx);

/* Fused form: *queued = the tiles the last fused step ran through the whole cycle (the
 * others it copied as at rest), *tiles = the tiles of the grid.  Synchronises.  Both 0
 * before the first fused step after a state change; SALEC_EORDER before salec_finalize. */
salec_status salec_fused_queue(salec_ctx* ctx, int* queued, int* tiles);

/* Per-kernel timing: with timing on, salec_step records a CUDA event before the first
 * and after every timed kernel of each step on the context's stream; salec_kernel_times
 * synchronises, returns in avg_ms[k] (n >= 6; unused entries 0) the mean duration of
 * kernel k over the steps recorded since timing was switched on or last read, the number
 * of steps in *steps, and restarts the count.  Phase form: k < 6 are the phases (phase 0
 * includes the Courant kernel); fused form: k = 0 the Courant and rest-tile kernels,
 * k = 1 the tile kernel; with the copy beside the tile kernel, k = 0 from before the
 * Courant kernel to the end of the copy kernel (second stream), k = 1 the tile kernel
 * alone (the two overlap).
 * salec_step_kernel_name(ctx, k) names entry k of the context's form ("" for an unused
 * one); salec_kernel_name(k) names phase k of the phase form. */
salec_status salec_set_kernel_timing(salec_ctx* ctx, int on);
salec_status salec_kernel_times(salec_ctx* ctx, double* avg_ms, int n, int* steps);
const char* salec_kernel_name(int k);
const char* salec_step_kernel_name(const salec_ctx* ctx, int k);

/* End time of a run (default: none).  salec_batch_run stops a run once t >= t_end; a
 * run at or past its end time, or whose status is not 0 (see salec_get_scalars), does
 * nothing in a batched step. */
salec_status salec_set_end_time(salec_ctx* ctx, double t_end);

/* Block shapes (threads in r x threads in z) of the six kernels of a step, as 12 ints
 * (x0, y0, ..., x5, y5).  x must be a multiple of 32, 128 <= x*y <= 512.  The shape changes
 * no field, only speed. */
salec_status salec_set_block_shapes(salec_ctx* ctx, const int* shapes);
salec_status salec_get_block_shapes(const salec_ctx* ctx, int* shapes);

/* Autotuner: runs trial_steps real steps (after one untimed step) with each candidate
 * block shape for all kernels, timing every kernel with CUDA events, and keeps for each
 * kernel its fastest shape (written to shapes_out, 12 ints, if not NULL).  The simulation
 * advances by (candidates x (trial_steps + 1)) steps, seven candidates. */
salec_status salec_autotune(salec_ctx* ctx, int trial_steps, int* shapes_out);

/* Batches: many independent runs (each a finalized context with its own state buffer,
 * all of one precision, material count and strength setting) advanced together: every
 * step is six launches for the whole batch, one block per (run, tile) entry of a work list,
 * each run with its own time step and its own end time.  The batch needs one caller-owned
 * device buffer of salec_batch_bytes() bytes (run parameter blocks and work lists).
 * salec_batch_run replays a CUDA graph of `chunk` steps until every run reaches its end
 * time or fails (status not 0), or max_steps steps; salec_batch_poll copies each run's
 * (t, dt, steps, status, t_end) into out[5 r .. 5 r + 4].  Streams: all batch work goes on the stream given here. */
typedef struct salec_batch salec_batch;
salec_status salec_batch_bytes(salec_ctx* const* runs, int nruns, size_t* bytes);
salec_status salec_batch_create(salec_ctx* const* runs, int nruns, void* dev_buf, size_t bytes, void* stream,
                                salec_batch** out);
salec_status salec_batch_step(salec_batch* batch, int nsteps);
salec_status salec_batch_run(salec_batch* batch, int chunk, long max_steps, long* steps_done, int* runs_done);
salec_status salec_batch_poll(salec_batch* batch, double* out);
salec_status salec_batch_autotune(salec_batch* batch, int trial_steps, int* shapes_out);

/* Persistent mode (on != 0; off is the default): each salec_batch_step call, and each
 * chunk of salec_batch_run (captured in its CUDA graph with the clearing of the barrier
 * word, or launched directly where the device refuses to capture it), is ONE cooperative
 * launch of a grid that the device holds at once.  Its blocks loop over the steps and, in
 * each, over the (run, tile) entries of every phase, with a grid-wide barrier between the
 * phases and a pass of per-run Courant steps after phase 0: the same code per cell and
 * vertex as the six launches per step, so the fields are bitwise those of the default
 * mode.  Every phase takes one block shape of at most 256 threads (the first kernel's,
 * else 32 x 4; salec_batch_autotune then picks one shape for all six).  Every barrier wait
 * is bounded (2 s); a wait that ran out ends the launch and the next salec_batch_poll or
 * salec_batch_run returns SALEC_ETIMEOUT.  SALEC_ECUDA when the kernel cannot be made
 * resident. */
salec_status salec_batch_set_persistent(salec_batch* batch, int on);

/* Failure detection, for testing it: the next salec_batch_step call (persistent mode)
 * starts its launch with the barrier's arrival counter far above the grid size, so no
 * block completes the first barrier (after phase 0 of the first step, which changes no
 * persistent field but the peak over-pressure, with the same values a repeat writes).
 * Every block's wait there runs out after 2 s and the launch ends; that step call's poll
 * returns SALEC_ETIMEOUT, and later steps continue from the unchanged state.  SALEC_EINVAL
 * outside persistent mode. */
salec_status salec_batch_expire_next_barrier(salec_batch* batch);
const char* salec_batch_last_error(const salec_batch* batch);
void salec_batch_destroy(salec_batch* batch);

/* Courant time step without any allocation, for callers that cannot allocate or lend
 * device memory (an external memory manager owns every allocation, a plug-in sees only
 * another program's field pointers, the allocator is locked).  The paper has no
 * counterpart; it is the step size salec_step's first kernel computes, evaluated on
 * caller-owned device buffers:
 *   grid    nr, nz, nmat, dx, cfl, dt_growth, dt_max, dt_min are used
 *   mats    nmat materials (host)
 *   fr[m]   device pointer to nr*nz (f_m, rho_m) pairs of doubles, row-major [j][i]
 *   I       device pointer to nr*nz specific internal energies
 *   D       device pointer to nr*nz damage values, or NULL (not needed for dt)
 *   v       device pointer to (nr+1)*(nz+1) (v_r, v_z) pairs
 *   dt_prev the previous step (growth limit); *dt_out receives the step (host).
 * Cells are taken as uniform squares of grid->dx (a grid given non-uniform sizes with
 * salec_set_spacing needs salec_step's own step).  The call enqueues a memset and one
 * kernel on `stream` and synchronises it.  It returns SALEC_EUNSTABLE, leaving *dt_out
 * alone, where salec_step's status word would report a failure: a NaN vertex speed or
 * sound speed, or a step below grid->dt_min.  Its scratch is file-scope device memory of
 * fixed size (65536 blocks of 32 x 8 cells, e.g. 4096 x 4096 cells; larger grids, and
 * grids of more than 65535 block rows, return SALEC_EINVAL) held by every device that
 * loads the library until the process exits.  The first call on a device looks up that
 * memory's address with the device current; make it before any stream capture, and do
 * not use the call across a device reset.  All calls share the scratch: calls that
 * overlap on the GPU (different streams or threads) race.  Failures without a context are
 * described by salec_last_error(NULL). */
salec_status salec_courant_dt_noalloc(const salec_grid* grid, const salec_material* mats,
                                      const double* const* fr, const double* I, const double* D,
                                      const double* v, double dt_prev, double* dt_out, void* stream);

/* Message of the last failure of `ctx`; with ctx == NULL, of the last failed call of this
 * thread that has no context. */
const char* salec_last_error(const salec_ctx* ctx);
void salec_destroy(salec_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* SALEC_H */
