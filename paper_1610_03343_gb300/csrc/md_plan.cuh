// md_plan.cuh -- host-side launch plan: every device buffer and size one context uses,
// plus the launch entry points implemented in neigh.cu and force.cu.
#pragma once

#include "md_internal.cuh"

namespace mdk {

struct Plan {
    int64_t N = 0;         // atoms (a pool: its atom capacity)
    // spatial decomposition: atoms [0, n_owned) are this rank's, the rest ghosts whose
    // positions another rank supplies -- ghosts take part in the list and the pair pass
    // (their neighbourhoods complete the owned atoms' forces) but are not integrated,
    // gathered or summed.  -1: every atom is owned.
    int64_t n_owned = -1;
    Box box{};             // box of the single system (pools: per-system boxes in `sys`)
    int kind = 0;          // 1 Tersoff, 2 SW
    int precision = 0;     // 0 fp64, 1 mixed
    int cap = 32;          // list capacity
    int maxa = 8;          // in-cutoff capacity (compact pair rows)
    double rc = 0, rl = 0, skin = 0;
    float list_margin = 0.f;   // fp32 margin of the list build
    // launch tuning (results do not depend on it): threads per block of the pair pass's
    // common-case launch (0 = default for the precision) and, for pools, blocks per SM of
    // the kernels that loop over the running systems' chunks
    int pair_block = 0;
    int pool_bps = 16;
    int pair_cap = 0;    // bond slots of the common-case Tersoff pass (0: default 4; 3)
    // fp64 single-element Tersoff: the common-case pass keeps f_C (4 bonds) instead of
    // deferring every atom with a bond in the switching region (set when those are many)
    bool pair_fc = false;
    int n_sm = 152;
    // parameter sets (a single system uses set 0)
    int n_sets = 1;
    TersoffP tp[kMaxSets]{};
    SWP sp[kMaxSets]{};
    int ntypes = 1;
    // multi-element Tersoff (one system, n_elem > 1 elements): constants of every ordered
    // element pair (a, b): radial parameters mixed, B scaled by chi_ab, angular and
    // bond-order parameters of element a; and their device copy in the pair pass's type
    bool multi = false;
    int n_elem = 1;
    TersoffP tpair[kMaxTypes][kMaxTypes]{};
    void *ttab = nullptr;
    double mass[kMaxTypes] = {0, 0, 0, 0};
    double inv_mass[kMaxTypes] = {0, 0, 0, 0};

    // pools: many systems over one flattened atom index
    bool batch = false;        // kernels look up each atom's system
    int n_sys = 1;             // system slots
    int seg_max = 1;           // system segments one gather block can hold
    int *sys_of = nullptr;     // N
    SysDev *sys = nullptr;     // n_sys (device)

    // per-atom state (fp64)
    double *pos = nullptr, *vel = nullptr, *force = nullptr, *pos_build = nullptr;
    double *u = nullptr, *w = nullptr, *j = nullptr;
    float *posf = nullptr;      // fp32 positions for the list build
    double *stage = nullptr;    // 3N scratch for wrapped output positions
    int *type = nullptr;
    // neighbour list
    int *nn = nullptr, *nl = nullptr;
    uint8_t *rev = nullptr;
    uint32_t *mask = nullptr;
    int *ovf_count = nullptr, *ovf_list = nullptr;   // deferred atoms of the pair pass
    // pair arrays, element type double (fp64) or float (mixed): dU_i/dr_ij as maxa x N
    // vectors (Vec4), bond vectors as 3 x maxa x N components
    void *pd = nullptr, *pr = nullptr;
    // cells (single system: nc; pools: per-system grids in `sys`)
    int nc[3] = {1, 1, 1};
    int64_t ncell = 1;
    int *cell_count = nullptr, *cell_start = nullptr, *cell_atoms = nullptr;
    uint8_t *occ = nullptr;     // single system: per-axis cell occupancy (nc0 + nc1 + nc2 flags)
    int *atom_cell = nullptr, *atom_rank = nullptr, *scan_blocks = nullptr;
    int64_t nscanb = 1;
    int *rb_plan = nullptr, *rb_sys = nullptr, *rb_chunks = nullptr;   // pool rebuild work lists
    int *act_plan = nullptr, *act_chunks = nullptr;   // pools: 128-atom chunks of the live systems
    int *stable_plan = nullptr, *stable_chunks = nullptr;   // pools: the live systems not rebuilding
    // Berendsen coupling (NPT): some system of the context is coupled; steps then scale
    // velocities, coordinates and boxes on the device, and kernels of a single system read
    // its box and cell grid from sys[0]
    bool npt = false;
    double *npt_totals = nullptr;   // n_sys x kNptExtra: K_aa (3), W_aa (3) of the last step
    // reductions
    double *partials = nullptr;
    int nb_gather = 1;
    double *totals = nullptr;   // n_sys x kNumPartials
    double *series = nullptr;   // rows x n_sys x 5
    Flags *flags = nullptr;
};

// md_api.cu: one parameter set of md_params into set idx of p (its cutoff in *rc), and the
// options that fix a plan's precision, list capacities, cutoff and skin (MD_ERR_ARG if bad).
md_status plan_params(const md_params *params, Plan &p, int idx, double *rc);
md_status plan_options(Plan &p, const md_options &opt, int kind, double rc);

// Kernel classes, for per-kernel timing.
enum KernelClass { KC_KICK_DRIFT = 0, KC_REBUILD, KC_PAIR, KC_GATHER, KC_REDUCE, KC_COUNT };
extern const char *kKernelClassNames[KC_COUNT];

// neigh.cu
int scan_block_elems();
// fp32 safety margin added to rl in the list build (covers coordinate rounding) for
// coordinates up to lmax.
float list_margin_for(double lmax, double rl);
// Wrap positions, build the cell list, the sorted Verlet list (cutoff rl, entries with
// image shifts) and the reverse-slot index, for every system whose rebuild is
// requested (a single system: always); clears the requests.  Returns the number of
// kernels launched.
int launch_rebuild(const Plan &p, cudaStream_t s);
// Request a rebuild where an atom moved more than skin/2 since the last build.
void launch_displacement_check(const Plan &p, cudaStream_t s);
// dst[a N + i] = positions of atoms [a0, a0 + n) wrapped into [0, L) on periodic axes.
void launch_wrap_copy(const Plan &p, cudaStream_t s, double *dst, int64_t a0, int64_t n);
// Per-axis cell occupancy of the single system's positions for the grid nc in `box`:
// occ[off_a + c] = 1 where an atom's cell coordinate along axis a is c (off_0 = 0,
// off_1 = nc0, off_2 = nc0 + nc1); the caller clears occ first.
void launch_axis_occupancy(const Plan &p, cudaStream_t s, const Box &box, const int nc[3], uint8_t *occ);

// force.cu
// Multi-element Tersoff: bytes of the device table of pair constants, and the table
// itself (host buffer of that size) from p.tpair in the precision of p.
size_t tersoff_table_bytes(const Plan &p);
void fill_tersoff_table(const Plan &p, void *host);
// Pair-pass block size in use (the tuned one, else the precision's default).
int effective_pair_block(const Plan &p);
bool valid_pair_block(int b);
int effective_pair_cap(const Plan &p);
// Opt the pair kernels into their dynamic shared memory on the current device (once per
// device); false if that failed.
constexpr int kMaxConfigDevices = 64;
bool configure_kernels(const Plan &p);
// Half-kick + drift + displacement check (first half of a velocity-Verlet step).
void launch_kick_drift(const Plan &p, cudaStream_t s, const double *half_kick, double dt);
// Start of a step: claim the series row, reset the pair pass's deferred count, count
// down per-system step budgets (pools) and set the rebuild conditional from
// flags->rebuild (h may be null when the graph has no rebuild node).
void launch_step_begin(const Plan &p, cudaStream_t s, const cudaGraphConditionalHandle *h);
// Pools: list the 128-atom chunks of the systems that run now (kick, pair and gather loop
// over this list, so a step costs in proportion to the atoms resident and running).
void launch_active_plan(const Plan &p, cudaStream_t s);
// Pools: list the chunks of the running systems that do not rebuild their list this step
// (taken after the kick's skin test), so that their pair pass need not wait for the
// rebuild of the others; sets the rebuild conditional h (may be null) when any running
// system is to be rebuilt or a rebuild was requested.
void launch_stable_plan(const Plan &p, cudaStream_t s, const cudaGraphConditionalHandle *h);
// Zero the pair pass's deferred-atom count (force evaluations outside a step).
void launch_pair_reset(const Plan &p, cudaStream_t s);
// Pools: mark every system as no longer fresh and end a fresh-only evaluation.
void launch_clear_fresh(const Plan &p, cudaStream_t s);
// Per-atom pair pass: U_i and dU_i/dr_ij for every in-cutoff neighbour.  Two launches:
// a pass whose shared-memory staging holds 4 bonds per atom (the crystals' common case),
// which defers any atom with more to a list, and a pass over that list with the full
// capacity.  Returns the number of kernels launched.
// Pools choose the atoms by chunk list: every running system (PAIR_ALL), those not
// rebuilding (PAIR_STABLE) or those just rebuilt (PAIR_REBUILT, the rebuild plan's list);
// `parts` selects the common-case launch (PAIR_FAST), the deferred atoms' launch
// (PAIR_DEFERRED) or both.  Single systems ignore the list.
enum { PAIR_ALL = 0, PAIR_STABLE = 1, PAIR_REBUILT = 2 };
enum { PAIR_FAST = 1, PAIR_DEFERRED = 2, PAIR_BOTH = 3 };
int launch_pair(const Plan &p, cudaStream_t s, int list = PAIR_ALL, int parts = PAIR_BOTH);
// Per-atom gather: F_i (Eq. 28), J_i (Eq. 30) and, for a force evaluation, W_i (Eq. 29)
// and per-atom outputs; optional half-kick (and per-system damping); block partials.
// fuse_next (a step followed by another in the same graph; not under NPT): also the next
// step's first half-kick, drift and skin test, so that step launches no k_kick_drift.
void launch_gather(const Plan &p, cudaStream_t s, const double *half_kick, double dt, bool full_outputs,
                   bool fuse_next = false);
int gather_block();
int gather_blocks(int64_t N);
// Fixed-order reduction of the gather's block partials into per-system totals (and a
// series row).
void launch_reduce(const Plan &p, cudaStream_t s, bool full_outputs, bool record_series);
// NPT, right after the kick of a step: scale the box edges of the coupled systems by the
// pending mu (the kick scaled velocities and coordinates), shrink cell grids that became
// too fine for the stencil, and clear the pending scaling.
void launch_npt_apply(const Plan &p, cudaStream_t s);
// NPT, at the end of a step: lambda and mu of each coupled system from the step's
// totals, left pending for the next step.
void launch_npt_couple(const Plan &p, cudaStream_t s, double dt);

}  // namespace mdk
