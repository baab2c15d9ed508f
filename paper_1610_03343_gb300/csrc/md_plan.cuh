// md_plan.cuh -- host-side launch plan: every device buffer and size one context uses,
// plus the launch entry points implemented in neigh.cu and force.cu.
#pragma once

#include "md_internal.cuh"

namespace mdk {

struct Plan {
    int64_t N = 0;
    Box box{};
    int kind = 0;          // 1 Tersoff, 2 SW
    int precision = 0;     // 0 fp64, 1 mixed
    int cap = 32;          // list capacity
    int maxa = 8;          // in-cutoff capacity (compact pair rows)
    double rc = 0, rl = 0, skin = 0;
    TersoffP tp{};
    SWP sp{};
    int ntypes = 1;
    double mass[kMaxTypes] = {0, 0, 0, 0};
    double inv_mass[kMaxTypes] = {0, 0, 0, 0};

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
    // pair arrays, element type double (fp64) or float (mixed)
    void *pd = nullptr, *pr = nullptr;
    // cells
    int nc[3] = {1, 1, 1};
    int64_t ncell = 1;
    int *cell_count = nullptr, *cell_start = nullptr, *cell_atoms = nullptr;
    int *atom_cell = nullptr, *atom_rank = nullptr, *scan_blocks = nullptr;
    int64_t nscanb = 1;
    // reductions
    double *partials = nullptr;
    int nb_gather = 1;
    double *totals = nullptr;   // kNumPartials
    double *series = nullptr;   // rows of 5
    Flags *flags = nullptr;
};

// Kernel classes, for per-kernel timing.
enum KernelClass { KC_KICK_DRIFT = 0, KC_REBUILD, KC_PAIR, KC_GATHER, KC_REDUCE, KC_COUNT };
extern const char *kKernelClassNames[KC_COUNT];

// neigh.cu
int scan_block_elems();
// fp32 safety margin added to rl in the list build (covers coordinate rounding).
float list_margin(const Plan &p);
// Wrap positions, build the cell list, the sorted Verlet list (cutoff rl, entries with
// image shifts) and the reverse-slot index; clears flags->rebuild.  Returns the number
// of kernels launched.
int launch_rebuild(const Plan &p, cudaStream_t s);
// Set flags->rebuild if any atom moved more than skin/2 since the last build.
void launch_displacement_check(const Plan &p, cudaStream_t s);
// dst[3N] = positions wrapped into [0, L) on periodic axes.
void launch_wrap_copy(const Plan &p, cudaStream_t s, double *dst);

// force.cu
size_t pair_smem_bytes(const Plan &p);
void configure_kernels(const Plan &p);
// Half-kick + drift + displacement check (first half of a velocity-Verlet step).
void launch_kick_drift(const Plan &p, cudaStream_t s, const double *half_kick, double dt);
// Start of a graph step: claim the series row and set the rebuild conditional from
// flags->rebuild (h may be null when the graph has no rebuild node).
void launch_step_begin(const Plan &p, cudaStream_t s, const cudaGraphConditionalHandle *h);
// Per-atom pair pass: U_i and dU_i/dr_ij for every in-cutoff neighbour.
void launch_pair(const Plan &p, cudaStream_t s);
// Per-atom gather: F_i (Eq. 28), J_i (Eq. 30) and, for a force evaluation, W_i (Eq. 29)
// and per-atom outputs; optional half-kick; block partial sums.
void launch_gather(const Plan &p, cudaStream_t s, const double *half_kick, bool full_outputs);
int gather_blocks(int64_t N);
// Fixed-order reduction of the gather's block partials into totals (and a series row).
void launch_reduce(const Plan &p, cudaStream_t s, bool full_outputs, bool record_series);

}  // namespace mdk
