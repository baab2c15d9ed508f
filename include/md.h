/*
 * md.h -- C ABI of the GB300 many-body MD library (libmd.so).
 *
 * Computes, for the Tersoff (Tersoff 1989) and Stillinger-Weber (Stillinger & Weber 1985)
 * potentials, the per-atom force, energy, virial and heat current in the explicit
 * pairwise-force form of Fan, Chen, Vierimaa, Harju, "Efficient molecular dynamics
 * simulations with many-body potentials on graphics processing units", CPC 2017
 * (arXiv:1610.03343), and integrates the motion with velocity Verlet (Sec. 3):
 *
 *   F_i = sum_j (dU_i/dr_ij - dU_j/dr_ji)                      (Eq. 28; Eqs. 12-14)
 *   W_i = -1/2 sum_j r_ij (x) (dU_i/dr_ij - dU_j/dr_ji)         (Eq. 29; Eq. 21)
 *   J_i = sum_j r_ij (dU_j/dr_ji . v_i)                        (Eq. 30; Eqs. 26-27)
 *   U_i = 1/2 sum_j U_ij                                       (Eqs. 1-2)
 *
 * with r_ij = r_j - r_i (Sec. 2.1, below Eq. 6), minimum image on periodic axes, and
 * (u (x) w)_ab = u_a w_b.  Units: Angstrom, eV, amu, fs; J in eV Angstrom/fs.
 *
 * Conventions for every call:
 *   - Every function returns md_status.  On failure the context keeps a message,
 *     readable with md_last_error(); the failing call leaves outputs undefined.
 *   - Input arrays are copied; the caller keeps ownership of every pointer it passes.
 *     Outputs are written into caller-owned buffers.
 *   - Pointers are host pointers unless md_options.io == MD_IO_DEVICE, in which case
 *     every array argument (positions, velocities, outputs; not box/pbc/params/totals/
 *     series) is a device pointer on the context's GPU.
 *   - Calls run on the context's CUDA stream and return after the results are in the
 *     caller's buffers (host I/O) or after the work is enqueued and synchronised
 *     (device I/O).
 *   - Arrays are SoA: a 3-vector field is 3N doubles (all x, then all y, then all z);
 *     a per-atom tensor is 9N doubles, component (a,b) at [(3a+b) N + i].
 *   - The box is orthorhombic with edges box[0..2]; a periodic axis needs
 *     box >= 2 (cutoff + skin), else MD_ERR_BOX (each pair then has one image).
 */
#ifndef MD_H
#define MD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct md_ctx md_ctx; /* opaque; owns all of its device memory */

typedef enum {
    MD_OK = 0,
    MD_ERR_ARG = -1,            /* bad argument (NULL where required, negative size, ...) */
    MD_ERR_BOX = -2,            /* periodic box shorter than 2 (cutoff + skin)            */
    MD_ERR_NEIGH_OVERFLOW = -3, /* an atom had more neighbours than max_neigh / max_active */
    MD_ERR_OOM = -4,            /* device allocation failed or exceeded hbm_budget        */
    MD_ERR_CUDA = -5,           /* a CUDA runtime call failed                             */
    MD_ERR_TIMEOUT = -6,        /* a bounded wait gave up (md_server_wait_timeout)        */
    MD_ERR_NAN = -7,            /* a non-finite force, position or velocity appeared      */
    MD_ERR_STATE = -8           /* call out of order (e.g. run before positions are set)  */
} md_status;

enum { MD_TERSOFF = 1, MD_SW = 2 };      /* md_params.kind */
enum { MD_FP64 = 0, MD_MIXED = 1 };      /* md_options.precision */
enum { MD_IO_HOST = 0, MD_IO_DEVICE = 1 }; /* md_options.io */

/* Potential parameters.
 *   MD_TERSOFF, n_types = 1: p[11] = A (eV), B (eV), lambda (1/A), mu (1/A), beta, n, c, d, h,
 *               R (A), S (A): Eqs. 2-6 with f_R = A exp(-lambda r), f_A = B exp(-mu r), and
 *               f_C = 1 (r < R), 1/2 + 1/2 cos(pi (r-R)/(S-R)) (R <= r < S), 0 (r >= S).
 *   MD_TERSOFF, n_types = T in 2..4 (md_create only; Sec. 2.1 closes by noting that the
 *               method covers systems of several elements): the multicomponent form of Tersoff, Phys.
 *               Rev. B 39, 5566 (1989).  p[11 T + T T] = T element rows of the 11 values
 *               above, then chi[a][b] row-major (each > 0).  A bond from an atom of element
 *               a to one of element b uses A_ab = sqrt(A_a A_b), B_ab = sqrt(B_a B_b),
 *               R_ab = sqrt(R_a R_b), S_ab = sqrt(S_a S_b), lambda_ab = (lambda_a +
 *               lambda_b)/2, mu_ab likewise; g and the bond order use element a's c, d, h,
 *               beta, n, and b_ij = chi_ab (1 + (beta_a zeta_ij)^n_a)^(-1/(2 n_a)), with
 *               zeta_ij = sum_k f_C^{a t_k}(r_ik) g_a(theta_ijk).  types[] are element rows.
 *   MD_SW:      p[9]  = epsilon (eV), sigma (A), a, lambda, gamma, A, B, p, q (n_types = 1)
 *               U_i = 1/2 sum_j phi2(r_ij) + sum_{j<k} phi3(r_ij, r_ik, theta_jik),
 *               the three-body term belonging to its vertex atom i.
 * The array is copied at md_create. */
typedef struct {
    int kind;
    int n_types;
    const double *p;
} md_params;

/* Options; fill with md_default_options() and override. */
typedef struct {
    int precision;     /* MD_FP64: all arithmetic in fp64.  MD_MIXED: per-pair bond-order
                          and derivative arithmetic in fp32; positions, velocities,
                          minimum-image displacements and system totals in fp64. */
    double skin;       /* Verlet skin (A); the list is rebuilt when an atom has moved more
                          than skin/2 since the last build (0 = default, 0.15 x cutoff). */
    int max_neigh;     /* list capacity per atom, <= 32 (default 32)                    */
    int max_active;    /* capacity of in-cutoff neighbours per atom, <= 16 (0 = default:
                          8 for one-element Tersoff; 16 for SW, whose second shell in
                          diamond Si sits only 0.07 A outside the cutoff, and for several
                          Tersoff elements, SiC's second Si-Si shell being as close)     */
    int io;            /* MD_IO_HOST (default) or MD_IO_DEVICE                           */
    void *cuda_stream; /* cudaStream_t to run on, or NULL: the context creates its own  */
    size_t hbm_budget; /* bytes the context may allocate; 0 = unlimited                 */
    int device;        /* CUDA device ordinal (default 0)                               */
} md_options;

/* Fill *opt with defaults (precision MD_FP64, skin 0 = default, max_neigh 32,
 * max_active 0 = default, host I/O, own stream, no budget, device 0). */
md_status md_default_options(md_options *opt);

/* Create a context for n_atoms atoms (n_atoms >= 0).
 *   box[3]  orthorhombic edge lengths (A), each > 0
 *   pbc[3]  1 = periodic along that axis, 0 = open
 *   types   n_atoms element indices < params->n_types (all 0 for a single element) -- host
 *           pointer always
 *   masses_by_type  params->n_types masses (amu), host pointer
 * MD_ERR_ARG for an index out of range, several elements with SW, or a bad parameter.
 * Positions and velocities start at zero; set them before computing. */
md_status md_create(md_ctx **out, const double box[3], const int pbc[3], int64_t n_atoms,
                    const int32_t *types, const double *masses_by_type,
                    const md_params *params, const md_options *opt);

/* Positions, SoA (x[N], y[N], z[N]), A.  Coordinates on periodic axes are wrapped into
 * [0, L).  Invalidates the neighbour list and forces.  (Pools: MD_ERR_STATE; systems
 * bring their positions to md_batch_add.) */
md_status md_set_positions(md_ctx *ctx, const double *x, const double *y, const double *z);

/* Velocities, SoA, A/fs. */
md_status md_set_velocities(md_ctx *ctx, const double *vx, const double *vy, const double *vz);

/* One force evaluation at the current positions and velocities (Algorithm 2's outputs):
 *   f [3N] forces (eV/A), u [N] per-atom energies (eV), w [9N] per-atom virials (eV),
 *   j [3N] per-atom potential heat currents (eV A/fs),
 *   totals[13] = U, W (9 components), J (3), summed in fp64 in a fixed order.
 * Any output pointer may be NULL (not requested).  totals is always a host pointer. */
md_status md_compute(md_ctx *ctx, double *f, double *u, double *w, double *j, double *totals);

/* Advance n_steps velocity-Verlet steps of dt_fs (NVE):
 *   v += F/m dt/2; x += v dt (wrapped); [rebuild list if needed]; F = F(x);
 *   v += F/m dt/2; record U, K, J with x(t+dt), v(t+dt).
 * series: NULL or n_steps x n_systems x 5 doubles (U, K, Jx, Jy, Jz per step and
 * system; n_systems = 1 for md_create contexts, max_systems for pools; host pointer, or
 * a device pointer under MD_IO_DEVICE).  Steps are replayed from CUDA graphs; the host
 * is not involved between steps. */
md_status md_run(md_ctx *ctx, int64_t n_steps, double dt_fs, double *series);

/* Current positions and velocities, each 3N SoA; either may be NULL. */
md_status md_get_state(md_ctx *ctx, double *x, double *v);

/* Checkpoint and resume (single-system contexts; pools: MD_ERR_STATE).  The paper has no
 * counterpart: it runs one uninterrupted simulation per benchmark (Sec. 3).  A checkpoint is
 * the whole state the next md_run step reads -- positions as stored (unwrapped since the
 * last list build), velocities, forces, build positions, the neighbour list and its reverse
 * slots, the box, cell grid and Berendsen state, and the pending rebuild request -- so a run
 * resumed from it in another context is bitwise identical to the uninterrupted run (no
 * atomics anywhere: every result depends only on that state).  md_get_state's wrapped
 * positions are not enough for that: a list built from them rounds differently.
 *   md_checkpoint_size: bytes of the image (header + about 96 + 13 cap bytes per atom).
 *   md_checkpoint_save: writes the image into a host buffer of at least that size.
 *   md_checkpoint_load: restores an image into a context created with the same atom count,
 *     types, masses, potential and options (precision, skin, list capacities); MD_ERR_ARG if
 *     the image is not a checkpoint, is truncated, or came from a different context. */
md_status md_checkpoint_size(md_ctx *ctx, size_t *bytes);
md_status md_checkpoint_save(md_ctx *ctx, void *buf, size_t bytes);
md_status md_checkpoint_load(md_ctx *ctx, const void *buf, size_t bytes);

/* Berendsen weak coupling (NPT).  The paper's benchmarks run in the NPT ensemble at 300 K
 * and 0 Pa (Sec. 3) without printing the coupling; this is Berendsen et al., J. Chem.
 * Phys. 81, 3684 (1984).  At the end of every md_run step, from that step's totals,
 *   T      = 2K / (k_B (3N - 3)),      lambda = sqrt(1 + dt/tau_T (T0/T - 1))  (0 if negative),
 *   P_aa   = (2 K_aa + W_aa) / V,      mu_a   = cbrt(1 - beta dt/tau_P (P0 - P_aa)),
 * with K_aa = sum_i m_i v_ia^2 / 2, W the total virial (the sum of the per-atom virials of
 * Eq. 29), V = Lx Ly Lz, P in GPa (1 eV/A^3 = 160.2176634 GPa).  The next step starts by
 * multiplying every velocity by lambda and every coordinate and box edge along a by mu_a
 * (mu_a = 1 on open axes, uncoupled axes, or tau_P <= 0; lambda = 1 for tau_T <= 0), then
 * takes its half-kick.  The scaling computed at the last step of a call stays pending and
 * is applied at the first step of the next md_run (so consecutive calls continue one
 * trajectory); md_set_positions drops it.  Everything runs on the device inside the
 * graph-replayed steps (the host is not involved between steps).
 *   system: 0 for md_create contexts; a pool's slot id.
 *   npt:    the coupling, or NULL to return the system to NVE (its list is then rebuilt).
 *           T0 >= 0, beta >= 0, all finite; couple[a] in {0, 1}.  Setting new constants on
 *           a coupled system keeps its pending scaling.
 * The box changes: md_get_box reads it.  The neighbour list stays exact: the skin test
 * allows for the scaling since the last build, and a cell grid whose cells became
 * narrower than the list radius is coarsened on the device.  A periodic edge that shrinks
 * below 2 (cutoff + skin) + 0.01 A makes md_run return MD_ERR_BOX.  MD_ERR_ARG for a bad
 * system or parameter. */
typedef struct {
    double T0;      /* bath temperature (K)                                  */
    double P0;      /* bath pressure (GPa), the same on every coupled axis   */
    double tau_T;   /* thermostat time constant (fs); <= 0: no thermostat    */
    double tau_P;   /* barostat time constant (fs); <= 0: no barostat        */
    double beta;    /* isothermal compressibility (1/GPa)                    */
    int couple[3];  /* 1: the barostat scales this (periodic) axis           */
} md_npt;
md_status md_set_npt(md_ctx *ctx, int system, const md_npt *npt);

/* Current box edges (A) of a system (0 for md_create contexts; a pool's slot id). */
md_status md_get_box(md_ctx *ctx, int system, double box[3]);

/* Counters for tests and benchmarks. */
typedef struct {
    int64_t n_atoms;
    int64_t steps_done;      /* MD steps since creation                               */
    int64_t n_rebuilds;      /* neighbour-list builds since creation                  */
    int max_neigh_seen;      /* largest list length at the last build                 */
    int kernel_launches_per_step; /* kernels of one md_run step launched on its own (inside
                                 a graph of steps, each step after the first has its first
                                 half-kick fused into the previous step's gather)         */
    int kernel_launches_per_rebuild; /* extra kernels of a step that rebuilds the list */
    int pair_deferred;       /* atoms with more in-cutoff bonds than the common-case pass
                                stages (Tersoff 4, SW 8; the fp64 single-element Tersoff
                                stagings also defer atoms with a bond in f_C's switching
                                region) at the last pair pass, handled by the
                                full-capacity pass (SW: one warp per atom)              */
    size_t device_bytes;     /* bytes the context has allocated on the device         */
    int64_t atoms_rebuilt;   /* atoms whose neighbour list was built, summed over builds
                                (pools: only the systems that needed a rebuild)          */
    int64_t kernels_launched; /* kernels md_run has launched (graph replays included; the
                                 kernels of taken list rebuilds are not counted: add
                                 kernel_launches_per_rebuild per rebuild)               */
} md_stats;
md_status md_get_stats(md_ctx *ctx, md_stats *out);

/* Launch mode of md_run.  use_graphs = 1 (default): steps are replayed from captured
 * CUDA graphs whose list rebuild is a conditional node decided on the device.
 * use_graphs = 0: the same kernels launched one by one, the rebuild decided on the host
 * after each drift (one small device-to-host copy per step); profilers that cannot
 * look inside graphs with conditional nodes see every kernel this way. */
md_status md_set_graph_mode(md_ctx *ctx, int use_graphs);

/* Launch tuning.  Three launch parameters are free choices that do not change any result
 * (every atom is computed by one thread the same way whatever they are; the gather's
 * partial sums are per 128-atom chunk, not per CUDA block), only the speed:
 *   pair_block          threads per block of the pair pass's common-case launch
 *                       (32, 64, 128 or 256; each thread stages one atom's bonds in shared
 *                       memory, so a block covers pair_block atoms);
 *   pool_blocks_per_sm  pools: blocks per SM of the kick, pair and gather kernels that
 *                       loop over the running systems' 128-atom chunks (1..64), i.e. how
 *                       many chunks (atoms / 128) one block takes on per step;
 *   pair_cap            bonds staged per atom by the common-case pass of a single-system
 *                       fp64 Tersoff context (one element): 3 or 4 (0 = 4).  Atoms with
 *                       more in-cutoff bonds go to the full-capacity pass, computed the same
 *                       way; 3 leaves room for more resident warps when most atoms have 3
 *                       bonds (the honeycomb sheet).  The fp64 single-element stagings
 *                       (3 or 4 bonds; pools: 4) keep no f_C values: an atom with a bond
 *                       in the switching region R <= r < S also goes to the full-capacity
 *                       pass.  When the last pair pass of an md_run call deferred more
 *                       than 1/16 of the atoms (a liquid, a hot amorphous state), the
 *                       context's later calls stage 4 bonds with f_C instead, and pair_cap
 *                       reads 4.  Other contexts stage 4 (Tersoff) or 8 (SW) whatever it
 *                       is.
 * md_autotune times each candidate on the context's current state with CUDA events on
 * its stream -- pair_block over {32, 64, 128, 256} (for each pair_cap where there is a
 * choice) with the pair pass alone, then (pools)
 * pool_blocks_per_sm over {4, 8, 16, 32, 64} with the pair pass and a gather without the
 * half-kick -- `repeats` launches each (0: 10), keeps the fastest and stores it in the
 * context; the next md_run captures its graphs with it.  The timed launches recompute the
 * current forces and change no state (positions, velocities, lists, step budgets).
 * Positions must be set (MD_ERR_STATE otherwise).  `out` (may be NULL) receives the
 * choice and every candidate's mean time.  md_set_tuning imposes a choice (MD_ERR_ARG for
 * values outside the sets above; pair_block 0 = the precision's default: 64 for
 * MD_FP64, 128 for MD_MIXED; pair_cap 0 = 4) and md_get_tuning reads the one in use.  The paper fixes
 * its block size by hand (Sec. 3); this tuner has no counterpart there. */
#define MD_TUNE_MAX 16
typedef struct md_tuning {
    int pair_block;
    int pool_blocks_per_sm;
    int n_tried;                      /* md_autotune: candidates timed                */
    int tried_pair_block[MD_TUNE_MAX];
    int tried_blocks_per_sm[MD_TUNE_MAX];
    double tried_ms[MD_TUNE_MAX];     /* mean ms of one timed launch sequence          */
    int pair_cap;                     /* 3 or 4 in use (read); 0, 3 or 4 (md_set_tuning) */
    int tried_pair_cap[MD_TUNE_MAX];
} md_tuning;
md_status md_autotune(md_ctx *ctx, int repeats, md_tuning *out);
md_status md_set_tuning(md_ctx *ctx, const md_tuning *t);
md_status md_get_tuning(md_ctx *ctx, md_tuning *out);

/* Per-kernel timing.  While enabled, md_run records CUDA events around each kernel
 * class of every step and accumulates their elapsed times; md_kernel_times returns, for
 * up to max_k classes, the name, the number of timed launches and the total ms. */
md_status md_set_profiling(md_ctx *ctx, int enable);
md_status md_kernel_times(md_ctx *ctx, int max_k, const char **names, int64_t *launches,
                          double *total_ms, int *n_out);

/* ---------------------------------------------------------------- pools ----------
 * A pool holds many independent systems (up to max_systems) over one flattened atom
 * index of `atom_capacity` atoms, stepped together by md_run: every kernel of a step
 * covers the whole pool in one launch, each atom using its system's box, cell grid and
 * parameter set; per-system totals are reduced separately.  Systems are added and
 * removed between calls (continuous batching), each with its own step budget: a
 * system stops on the device when its budget reaches zero, so systems of different
 * lengths share the same graph-replayed steps.  A system's results are those it would
 * have alone (same kernels, same per-atom arithmetic and summation order).
 * All systems of a pool use one potential kind (Tersoff or SW); n_sets parameter sets
 * (elements) of that kind, one per system; per-atom types index masses_by_type.
 * Each system's atom range starts on a 128-atom boundary (a gather block never mixes
 * systems). */
typedef struct {
    double max_box;         /* largest box edge any system will have (A); 0 = 4096        */
    int64_t cell_capacity;  /* cells shared by all systems' grids; 0 = 4 x atom_capacity   */
} md_batch_options;

typedef struct {
    double box[3];          /* orthorhombic edges (A)                                   */
    int pbc[3];             /* periodic axes                                            */
    int64_t n_atoms;        /* >= 1                                                     */
    const int32_t *types;   /* n_atoms element indices < n_types (host pointer)          */
    int param_set;          /* index into the pool's parameter sets                     */
    const double *x, *y, *z;      /* positions, SoA (host or device per options.io)     */
    const double *vx, *vy, *vz;   /* velocities, or NULL for zero                        */
    int64_t n_steps;        /* steps to run before stopping (< 0: until removed)         */
    double damp;            /* damped-MD friction gamma (1/fs): v <- v (1 - gamma dt)
                               after each step (0 = NVE)                                 */
} md_system;

md_status md_batch_create(md_ctx **out, int64_t atom_capacity, int max_systems, int n_sets,
                          const md_params *param_sets, int n_types, const double *masses_by_type,
                          const md_batch_options *bopt, const md_options *opt);

/* Add a system (copies its arrays); *id receives its slot.  MD_ERR_OOM when the pool has
 * no free slot, atom range or cell range (admission can retry after removals). */
md_status md_batch_add(md_ctx *ctx, const md_system *sys, int *id);

/* Remove a system and free its slot, atoms and cells. */
md_status md_batch_remove(md_ctx *ctx, int id);

/* Per slot (max_systems entries each, any pointer may be NULL): active (1 running, 0
 * stopped, -1 empty slot), steps left, totals (13 per slot: U, W(9), J(3) of the last
 * step or force evaluation) and kinetic energy K of the last step. */
md_status md_batch_status(md_ctx *ctx, int *active, int64_t *steps_left, double *totals, double *kinetic);

/* Per slot (max_systems entries): MD_OK, or the md_status of the failure that stopped
 * that system on the device -- MD_ERR_NAN (a non-finite force, position or velocity),
 * MD_ERR_NEIGH_OVERFLOW (an atom with more than max_neigh listed or max_active in-cutoff
 * neighbours), MD_ERR_BOX (NPT: an edge shrank below 2 (cutoff + skin)).  Such a failure
 * concerns one system: it stops (md_batch_status reports it inactive) while md_run goes on
 * with the others and returns MD_OK; the caller removes it.  Empty slots read MD_OK.
 * md_batch_add with host I/O rejects non-finite positions or velocities itself (MD_ERR_NAN). */
md_status md_batch_errors(md_ctx *ctx, int *status);

/* Positions (wrapped) and velocities of one system, each 3 n_atoms SoA. */
md_status md_batch_get_state(md_ctx *ctx, int id, double *x, double *v);

/* ---------------------------------------------------------------- serving -------
 * A request loop over pools (continuous batching).  Jobs are submitted from any
 * thread at any time; each potential kind has a pool driven by its own host thread,
 * which admits queued jobs (first fit into the pool's free atom and cell ranges: the
 * job's device footprint; a job that does not fit lets later jobs pass for up to half a
 * second, then holds the queue until it fits), steps all admitted jobs together in
 * graph-replayed chunks,
 * and harvests jobs whose step budget ran out on the device (final state copied into
 * the job's output buffers, slot freed).  Jobs arriving while others run are admitted
 * as slots free up; the pools of different kinds run on their own streams and overlap
 * on the device.  A job's result equals that of the same system run alone. */
typedef struct md_server md_server;

typedef struct {
    int precision;              /* MD_FP64 or MD_MIXED                                     */
    int64_t tersoff_atoms;      /* atom capacity of the Tersoff pool (0: no Tersoff jobs)   */
    int64_t sw_atoms;           /* atom capacity of the SW pool (0: no SW jobs)             */
    int max_jobs_per_pool;      /* system slots per pool                                   */
    double tersoff_dt, sw_dt;   /* time step of each pool (fs)                             */
    int chunk_steps;            /* steps per scheduling round (default 8)                  */
    int device;
} md_server_options;

typedef struct {
    int kind;                   /* MD_TERSOFF or MD_SW                                     */
    int param_set;              /* Tersoff: 0 = Si, 1 = C (md_server_create's sets); SW: 0  */
    double box[3];
    int pbc[3];
    int64_t n_atoms;
    const int32_t *types;       /* element indices (Tersoff: 0 Si, 1 C), copied at submit  */
    const double *x, *y, *z, *vx, *vy, *vz;  /* host SoA arrays, copied at submit         */
    int64_t n_steps;            /* >= 1                                                    */
    double damp;                /* 0: NVE; > 0: damped relaxation                          */
    double *x_out, *v_out;      /* host 3 n_atoms SoA buffers for the final state, or NULL;
                                   must stay valid until the job is done                  */
} md_job;

typedef struct {
    int done;                   /* 1 when finished (results written)                       */
    int status;                 /* MD_OK, or the error that failed the job                 */
    double t_submit, t_admit, t_done;  /* seconds on the server's monotonic clock          */
    double U, K;                /* final potential and kinetic energy (eV)                 */
} md_job_result;

typedef struct {
    int64_t submitted, admitted, completed, failed;
    double atom_steps;          /* atom-steps of completed jobs                            */
    double busy_seconds;        /* wall time with at least one job admitted (per pool, summed) */
    double run_seconds;         /* time inside md_run chunks (per pool, summed)            */
    double admit_seconds;       /* time admitting jobs                                     */
    double harvest_seconds;     /* time reading back and removing finished jobs            */
    int64_t chunks;             /* scheduling rounds                                       */
    double resident_atom_steps; /* atoms resident in the pools x chunk steps (incl. jobs that
                                   stopped inside a chunk)                                  */
} md_server_stats;

/* tersoff_sets: 2 parameter sets (Si, C) and masses (Si, C); sw_set: 1 set, its mass. */
md_status md_server_create(md_server **out, const md_server_options *opt, const md_params *tersoff_sets,
                           const double *tersoff_masses, const md_params *sw_set, const double *sw_mass);
/* Queue a job (thread-safe, returns at once); *job_id identifies it. */
md_status md_server_submit(md_server *srv, const md_job *job, int64_t *job_id);
/* Current state of a job (done = 0 while queued or running). */
md_status md_server_poll(md_server *srv, int64_t job_id, md_job_result *out);
/* Block until the job is done. */
md_status md_server_wait(md_server *srv, int64_t job_id, md_job_result *out);
/* Block until the job is done or timeout_s seconds have passed: MD_OK (done; *out holds
 * the result) or MD_ERR_TIMEOUT (not done yet; *out holds its state so far, done = 0).  For
 * callers with a deadline; the job keeps running either way. */
md_status md_server_wait_timeout(md_server *srv, int64_t job_id, double timeout_s, md_job_result *out);
/* Block until every submitted job is done. */
md_status md_server_drain(md_server *srv);
md_status md_server_stats_get(md_server *srv, md_server_stats *out);
/* Seconds since md_server_create on the server's monotonic clock (the job timestamps). */
double md_server_clock(const md_server *srv);
/* Finishes the jobs already submitted, stops the pool threads and frees the pools. */
void md_server_destroy(md_server *srv);

/* ------------------------------------------------------ spatial decomposition --------
 * One system split over ranks (processes, typically one GPU each) in slabs along one
 * periodic axis.  The paper runs a system on one GPU and compares with LAMMPS's MPI runs
 * (Sec. 3); splitting needs a halo because dU_j/dr_ji of an owned atom's neighbour j depends
 * on j's own neighbours (Eqs. 14, 28).  Rank r owns the atoms whose coordinate along `axis`
 * (wrapped into [0, L)) lies in [r L/n, (r+1) L/n) and keeps as ghosts every atom within
 * G = 2 (cutoff + skin + fp32 list margin) + 0.01 A of its slab, so it computes the
 * derivatives of its first-shell ghosts itself; ghosts are neither integrated nor summed.
 * Slabs must be at least 2G wide (MD_ERR_BOX).  Results equal the undivided system's up to
 * summation order (bonds are taken in another order).
 *
 * The library packs and unpacks messages; the caller moves them between ranks (any
 * transport: host-staged sockets, MPI, NCCL).  Each rank sends one message to its left
 * neighbour (rank - 1 mod n) and one to its right (rank + 1 mod n) and passes md_domain_unpack
 * the message its left neighbour sent right and the one its right neighbour sent left.
 * Message kinds (mode):
 *   MD_DOMAIN_POSITIONS  the current positions of the atoms the neighbour keeps as ghosts
 *                        (every step without a rebuild);
 *   MD_DOMAIN_MIGRATE    atoms whose slab changed (id, element, position, velocity);
 *   MD_DOMAIN_GHOSTS     the new ghost sets (id, element, position), after a migration.
 * A step of velocity Verlet (every rank, in this order):
 *   md_domain_kick_drift(dt, &r)   first half-kick and drift of the owned atoms; r = 1 when
 *                                  an owned atom moved more than skin/2 since the last build
 *   r = OR of r over the ranks (the caller's reduction)
 *   r == 0: exchange MD_DOMAIN_POSITIONS
 *   r == 1: exchange MD_DOMAIN_MIGRATE, then MD_DOMAIN_GHOSTS (the list is then rebuilt)
 *   md_domain_force(dt, totals)    forces, second half-kick; totals of the owned atoms (U, K,
 *                                  Jx, Jy, Jz), which the caller sums over the ranks
 * Start: md_domain_set_atoms (every rank may pass all atoms: each keeps its slab's), exchange
 * MD_DOMAIN_GHOSTS, then md_domain_force(0) for the first forces.  Single element only. */
typedef struct md_domain md_domain;
enum { MD_DOMAIN_POSITIONS = 0, MD_DOMAIN_MIGRATE = 1, MD_DOMAIN_GHOSTS = 2 };

/* Rank `rank` of `n_ranks` (>= 2); pbc[axis] must be 1; `capacity` bounds owned + ghost
 * atoms on this rank (device memory is sized for it; MD_ERR_OOM when exceeded). */
md_status md_domain_create(md_domain **out, const double box[3], const int pbc[3], int axis, int n_ranks, int rank,
                           int64_t capacity, const md_params *params, const double *masses_by_type,
                           const md_options *opt);
/* Atoms (host arrays; ids unique over the system, types all 0; velocities may be NULL). */
md_status md_domain_set_atoms(md_domain *dom, int64_t n, const int64_t *ids, const int32_t *types,
                              const double *x, const double *y, const double *z, const double *vx,
                              const double *vy, const double *vz);
/* Largest message this rank may send next in each direction, in bytes. */
md_status md_domain_message_bound(md_domain *dom, int mode, size_t *bytes);
/* Writes the two messages of kind `mode` (each buffer at least the bound) and their sizes. */
md_status md_domain_pack(md_domain *dom, int mode, void *to_left, void *to_right, size_t capacity,
                         size_t *n_left, size_t *n_right);
/* Takes the left neighbour's right-going and the right neighbour's left-going message;
 * MD_ERR_ARG for a message of another kind or one that does not match the ghost sets. */
md_status md_domain_unpack(md_domain *dom, int mode, const void *from_left, size_t n_left,
                           const void *from_right, size_t n_right);
md_status md_domain_kick_drift(md_domain *dom, double dt_fs, int *rebuild);
/* Forces on the owned atoms; dt_fs != 0 also applies the second half-kick. */
md_status md_domain_force(md_domain *dom, double dt_fs, double totals[5]);
/* One force evaluation with per-atom outputs of the owned atoms, in md_domain_owned's order
 * (host arrays: f 3n, u n, w 9n, j 3n SoA; any may be NULL) and the rank's totals[13]. */
md_status md_domain_compute(md_domain *dom, double *f, double *u, double *w, double *j, double totals[13]);
/* Owned atoms: count, ids (ascending), positions (wrapped, 3n SoA), velocities (3n SoA);
 * any array may be NULL. */
md_status md_domain_owned(md_domain *dom, int64_t *n, int64_t *ids, double *x, double *v);
const char *md_domain_last_error(const md_domain *dom);
void md_domain_destroy(md_domain *dom);

/* ------------------------------------------------------ allocation-free evaluation --
 * The paper has no counterpart to this entry point; it exists for callers that cannot
 * allocate device memory when they need forces (code running inside another runtime's
 * allocator or memory-pool callback, plugins whose host forbids allocation after
 * start-up, hosts that plan their whole device footprint in advance).
 *
 * md_compute_static is md_compute without a context: one force evaluation of one system
 * (F, U, W, J per atom and the 13 totals, the same kernels and results), using as scratch
 * a single file-scope device array of MD_STATIC_SCRATCH_BYTES that every GPU loading the
 * library holds until the process exits.  It calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *   - kind, params: as md_params (one element); mass in amu; precision MD_FP64/MD_MIXED.
 *   - x, y, z: device arrays of n_atoms positions; vx, vy, vz: device velocities or NULL
 *     (zero); f [3N], u [N], w [9N], j [3N]: device outputs, any may be NULL; totals: host
 *     array of 13 (U, W, J) or NULL.  Runs on cuda_stream (NULL: the default stream) and
 *     returns after synchronising it.
 *   - Sizes: n_atoms <= MD_STATIC_MAX_ATOMS, else MD_ERR_OOM (no work done); MD_ERR_OOM
 *     also when the cell grid would not fit (the grid is capped at 4 n + 64 cells).
 *   - The first call on a device resolves the array's device address with that device
 *     current; make that first call before any stream capture.
 *   - Every call reuses the same array and it keeps the previous call's contents (each
 *     call clears what must start at zero).  Calls that overlap on the GPU race on it:
 *     serialise them. */
#define MD_STATIC_SCRATCH_BYTES (16u << 20)
#define MD_STATIC_MAX_ATOMS 12288
md_status md_compute_static(int kind, const double *params, int precision, const double box[3],
                            const int pbc[3], int64_t n_atoms, const double *x, const double *y,
                            const double *z, const double *vx, const double *vy, const double *vz,
                            double mass, double *f, double *u, double *w, double *j, double *totals,
                            void *cuda_stream);

/* Green-Kubo transport from the heat current.  The paper derives the potential part of
 * the heat current for many-body potentials (Sec. 2.3, Eq. 30) for thermal-conductivity
 * work but does not print the Green-Kubo relation; this uses the textbook one on the
 * total J that md_run records every step:
 *   acf[m*3 + a]   = C_a(m) = 1/(T-m) sum_{t=0}^{T-m-1} J_a(t) J_a(t+m),  m < n_lags,
 *                    a = x, y, z (every time origin of the T = n_rows rows);
 *   kappa[m*3 + a] = 1/(k_B T^2 V) * trapezoid integral of C_a over lags 0..m with step
 *                    dt_fs, in W/(m K) (J in eV A/fs, V = volume in A^3, T = temperature
 *                    in K; kappa[0] = 0).
 * Layout: J_x of row t at j[t*row_stride], J_y at +1, J_z at +2.  For md_run's series
 * pass j = series + 2 with row_stride 5 (one system) or series + 5 s + 2 with row_stride
 * 5 n_systems (system s of a pool).  io: MD_IO_HOST (host arrays; copied through
 * stream-ordered device scratch) or MD_IO_DEVICE (device arrays).  kappa may be NULL
 * (then dt_fs, volume and temperature are not used).  Runs on cuda_stream and returns
 * after synchronising it; fp64 throughout, fixed summation order (deterministic).
 * Errors: MD_ERR_ARG for NULL j/acf, n_rows < 1, n_lags outside 1..n_rows, row_stride < 3,
 * or non-positive dt/volume/temperature with kappa requested; MD_ERR_CUDA otherwise. */
md_status md_hcacf(const double *j, int64_t n_rows, int64_t row_stride, int64_t n_lags, double dt_fs,
                   double volume, double temperature, double *acf, double *kappa, int io,
                   void *cuda_stream);

/* Diagnostics for accuracy tests: evaluates, on the current CUDA device, the fp64 routines
 * that the pair passes use in place of the CUDA math library: the table-driven exponential
 * (fn = 0) or logarithm (fn = 1) (P. T. P. Tang's table-driven method; exp within 2 ulp for
 * |x| <= 708, log to about 1e-16 (1 + |binary exponent of x|) absolute for positive normal
 * x), the reciprocal (fn = 2: fp32 seed and one third-order step, within 1 ulp for
 * 1.2e-38 < |x| < 8.5e37) or the reciprocal square root (fn = 3: fp32 seed and one
 * third-order step, within 1 ulp for 1.2e-38 < x < 3.4e38; +inf for x < 2^-126, so that a
 * zero-length bond between coincident atoms makes the forces non-finite, MD_ERR_NAN), and the
 * exponential (fn = 4) and logarithm (fn = 5) that the pair passes call: the same tables and
 * bounds, the range reduction and final multiply-add in fp64 and the correction polynomial
 * as pairs of floats on the fp32 pipe (three fp64 instructions each); the reciprocal (fn = 6)
 * and reciprocal square root (fn = 7) whose last step runs as float pairs (two fp64
 * instructions each); and the exponential (fn = 8; error about 2^-47 e^x + 2^-126 for
 * -80 <= x <= 80, x clamped to that range) and logarithm (fn = 9; absolute error about
 * 2^-47 (1 + |log x|) for 2^-78 <= x < 2^127) of the bond-order chain, which run on the
 * fp32 pipe alone: x is split into a float pair and the float-pair result summed back.
 * x, y: n host doubles.  Returns 0, -1 for bad arguments, -5 on a CUDA error.
 * Allocates and frees its own device scratch. */
int md_fastmath_eval(int fn, int64_t n, const double *x, double *y);

/* Diagnostics for rooflines: the fused multiply-add peak of the current device in fp64
 * (precision = MD_FP64) or fp32 (MD_MIXED), measured -- the paper's hardware figures
 * (Sec. 3) are a vendor's, this is what the GPU at hand delivers.  A kernel of independent
 * FMA chains (8 per thread in fp64, 16 in fp32; 1024 threads per SM on every SM; `iters`
 * FMAs per chain) runs `repeats` times after a warm-up launch, each timed with CUDA events;
 * *tflops receives the best rate (2 flop per FMA, TFLOP/s) and *ms (may be NULL) that
 * launch's time.  Allocates
 * and frees a small output buffer.  MD_ERR_ARG for iters < 1, repeats < 1 or another
 * precision. */
int md_peak_flops(int precision, int64_t iters, int repeats, double *tflops, double *ms);

/* Message of the last failing call (empty string if none).  Never NULL. */
const char *md_last_error(const md_ctx *ctx);

/* Free the context and all of its device memory.  NULL is accepted. */
void md_destroy(md_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* MD_H */
