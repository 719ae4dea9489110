/*
 * mdgb.h - C ABI of the GB300 (sm_103a) short-range molecular-dynamics hot path.
 *
 * The calls follow the problem statement of R. Meyer, "Efficient
 * Parallelization of Short-Range Molecular Dynamics Simulations on Many-Core
 * Systems" (arXiv:1305.4196): N particles in a periodic box whose
 * interactions vanish beyond a cutoff r_cut (Sec. I), binned into linked
 * cells at least as wide as the interaction range (Sec. II.A, step 1 of the
 * algorithm), neighbour lists built per cell (Sec. II.A), forces computed per
 * cell task (Sec. II.A, step 2) with no particle written by two workers at
 * once (Sec. II.A; Sec. II.B waves), thread-local energy accumulators and a
 * particle-parallel integration loop (Sec. II.C).
 *
 * Conventions shared by every call
 *  - Status: every int-returning call returns MD_OK (0) or a negative MD_ERR_*
 *    code; md_last_error() gives a message.  No exception or abort crosses the
 *    ABI.  A failed call leaves the system usable unless it returns MD_ERR_CUDA.
 *  - Atom order at the boundary is always the caller's original order
 *    (index 0..N-1 as passed to md_set_state); the library reorders atoms into
 *    cell order internally and hides it.
 *  - Arrays of 3-vectors are N x 3, row-major (x0 y0 z0 x1 y1 z1 ...).
 *  - Ownership: the caller owns every array it passes and keeps ownership;
 *    the library copies in or out during the call (stream-ordered) and owns
 *    only its opaque workspace, freed by md_destroy().
 *  - Host or device: calls with a `device_ptrs` argument take device pointers
 *    when it is non-zero and host pointers otherwise.  Everything runs on the
 *    CUDA stream given in md_params.stream (NULL: the legacy default stream)
 *    on the device that was current at md_create().
 *  - Calls are asynchronous on the stream except those that return host
 *    values (md_energy_virial, md_get_neighbors, md_get_info, host-pointer
 *    copies), which synchronise the stream before returning.
 *  - Units: reduced LJ units (sigma, epsilon, mass, tau).
 */
#ifndef MDGB_H
#define MDGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes */
#define MD_OK                 0
#define MD_ERR_ARG           -1  /* bad argument (null, size, range, species id) */
#define MD_ERR_BOX_TOO_SMALL -2  /* some box side < 4 (r_cut + skin): cell grid and minimum image invalid */
#define MD_ERR_CELL_OVERFLOW -3  /* a cell neighbourhood does not fit the on-chip tile even after regrowth */
#define MD_ERR_LIST_OVERFLOW -4  /* a neighbour list does not fit even after regrowth */
#define MD_ERR_NONFINITE     -5  /* a non-finite force or position appeared */
#define MD_ERR_SKIN_VIOLATION -6 /* fixed-interval rebuild policy and an atom moved more than skin/2 */
#define MD_ERR_CUDA          -7  /* a CUDA runtime call failed; the system should be destroyed */
#define MD_ERR_TIMEOUT       -8  /* a bounded device-side wait gave up */
#define MD_ERR_STATE         -9  /* call out of order (e.g. no md_set_state yet) */

/* ---- md_params.precision */
#define MD_FP64  0  /* FP64 positions, pair arithmetic and accumulation */
#define MD_MIXED 1  /* FP32 pair arithmetic, 64-bit fixed-point force sums, FP64 integration and reductions */

/* ---- md_params.list_kind */
#define MD_LIST_FULL         0  /* every pair in both atoms' lists; each list owned by one thread, no writes to j */
#define MD_LIST_HALF_COLOUR8 1  /* each pair once (Newton's third law); forces in 8 colour phases of 2x2x2-cell blocks */
/* Each pair once, and the forces evaluated with no atomic operation: the 8 colour phases of
 * blocks (Sec. II.B waves), inside a block 14 phases over
 * the half shell (the cell, then its 13 forward cells; Sec. II.D.3) separated by barriers,
 * in which the 8 cells of the block write 8 different cells, and inside a cell's warp a
 * schedule whose every step names distinct target atoms - the rule of Sec. II.A that no
 * particle is updated by two workers at once, down to the threads.  (A kernel that finds a
 * fault sets an error bit atomically, and the list build sums its statistics with one atomic
 * per warp; neither touches a force.)  MD_MIXED only; cells of at most 63 atoms (a denser
 * cell returns MD_ERR_CELL_OVERFLOW). */
#define MD_LIST_HALF_ATOMIC_FREE 2

/* ---- md_params.rebuild */
#define MD_REBUILD_SKIN_HALF 0  /* rebuild when some atom moved more than skin/2 since the last build (default) */
#define MD_REBUILD_EVERY_K   1  /* rebuild every rebuild_k steps, as in the paper's benchmarks (Sec. III) */

typedef struct md_system md_system; /* opaque; owns all device workspace */

typedef struct {
    int32_t n_species;     /* >= 1 */
    const double *eps;     /* n_species^2, row-major, symmetric: LJ well depth per species pair */
    const double *sigma;   /* n_species^2, row-major, symmetric: LJ diameter per species pair */
    const double *rcut;    /* n_species^2 or NULL: per-pair cutoff (NULL: r_cut of md_create for all pairs) */
    const double *mass;    /* n_species */
    double dt;             /* time step */
    int32_t precision;     /* MD_FP64 | MD_MIXED */
    int32_t list_kind;     /* MD_LIST_FULL | MD_LIST_HALF_COLOUR8 | MD_LIST_HALF_ATOMIC_FREE */
    int32_t rebuild;       /* MD_REBUILD_SKIN_HALF | MD_REBUILD_EVERY_K */
    int32_t rebuild_k;     /* interval for MD_REBUILD_EVERY_K */
    void *stream;          /* cudaStream_t, or NULL for the legacy default stream */
} md_params;

typedef struct {
    int64_t n;             /* atoms */
    int32_t ncell[3];      /* cells per dimension (multiples of 4; full lists also other even counts >= 6) */
    int32_t list_cap;      /* current neighbour-list capacity per atom */
    int32_t tile_cap;      /* current on-chip tile capacity (atoms of a 4x4x4-cell neighbourhood) */
    int64_t n_builds;      /* neighbour-list builds so far */
    int64_t n_steps;       /* time steps integrated so far */
    int64_t list_entries;  /* sum of list lengths at the last build */
    int32_t max_list;      /* longest list at the last build */
    int32_t max_tile;      /* largest tile at the last build */
    double cell_width[3];  /* sigma */
    int64_t kernel_launches;   /* kernels launched by the library so far */
    int64_t force_evals;       /* force evaluations (one per step, plus md_forces / md_energy_virial) */
    double force_ms;           /* summed device time of force evaluations (only while timing is on) */
    int64_t timed_force_evals; /* force evaluations included in force_ms */
    double build_ms;           /* summed device time of binning + list builds (only while timing is on) */
    int64_t timed_builds;      /* builds included in build_ms */
    int64_t n_redos;           /* md_step chunks redone after a rebuild outgrew the captured capacities */
} md_info;

/*
 * Create a system of n atoms in the periodic box box[3] (sides, sigma) with
 * cutoff r_cut and Verlet skin `skin` (neighbour-list radius r_cut + skin;
 * Sec. II.A).  Picks the cell grid: per dimension the largest multiple of 4
 * cells whose width is at least r_cut + skin (Sec. II.A: cells wider than the
 * interaction range; multiples of 4 so that 2x2x2-cell blocks split into 8
 * colour classes, Sec. II.D.2 blocking).  MD_LIST_FULL needs no colour classes
 * and takes 6 cells on a side where 6 fit but the rule gives 4, so that the
 * 4x4x4-cell neighbourhood of a block is not the whole box.  At least 4 cells
 * per side.  A Lennard-Jones system on the mixed full-list path then takes coarser
 * cells once, at its first build after md_set_state, never more of them: per side the
 * smallest even count (at least 6) whose width is at most (A / (8 rho))^(1/3),
 * so that a 2x2x2-cell block holds about A atoms for the force kernel's 256
 * threads.  Homogeneous systems (every block occupied, largest tile within 1.25x
 * the mean) take A = 224 and rho = N / V (44 -> 42 cells per side for
 * 2,048,000 atoms at rho* = 0.8442); others A = 200 and rho = the density the
 * average atom sees at the first grid (sum of squared cell counts / N / cell
 * volume).  MDGB_FIT_GRID=1 in the environment at md_create keeps the first
 * grid.  md_get_info reports the grid in use.  Allocates all device workspace.
 * Errors: MD_ERR_ARG, MD_ERR_BOX_TOO_SMALL, MD_ERR_CUDA.  *out is NULL on error.
 */
int md_create(int64_t n, const double box[3], double r_cut, double skin,
              const md_params *p, md_system **out);

/*
 * Load positions, velocities (N x 3, original order) and species ids (N,
 * values in [0, n_species); NULL: all 0).  Positions may lie anywhere; they
 * are mapped into [0, L) at the next neighbour build.  Invalidates forces and
 * lists.  Errors: MD_ERR_ARG (bad species id), MD_ERR_NONFINITE (a position
 * or velocity is NaN or infinite; the state is not loaded), MD_ERR_CUDA.
 */
int md_set_state(md_system *s, const double *pos, const double *vel,
                 const int32_t *species, int device_ptrs);

/*
 * Bin atoms into the cell grid (Sec. II.A, step 1): map positions into
 * [0, L) (updating image counters), assign each atom its cell, counting-sort
 * atoms into cell order (cells grouped by 2x2x2 block, atoms inside a cell in
 * original-index order) and reorder all per-atom state.  Invalidates lists.
 */
int md_bin_cells(md_system *s);

/*
 * Bin (as md_bin_cells) and build the neighbour lists (Sec. II.A): for each
 * atom every other atom at minimum-image distance < r_cut + skin, exactly the
 * set the FP64 definition gives at the current positions.  Records the
 * positions as the reference for the skin/2 displacement test.
 * Errors: MD_ERR_CELL_OVERFLOW / MD_ERR_LIST_OVERFLOW only if regrowth fails.
 */
int md_build_neighbors(md_system *s);

/*
 * Forces at the current positions (Sec. II.A, step 2), rebuilding the lists
 * first if there are none or some atom moved more than skin/2.  If f_out is
 * non-NULL the forces are copied to it (N x 3 doubles, original order).
 */
int md_forces(md_system *s, double *f_out, int device_ptrs);

/*
 * Integrate n_steps velocity-Verlet steps: v += dt F/(2m); x += dt v;
 * rebuild lists if the policy says so; F = F(x); v += dt F/(2m).
 * Steps run as CUDA-graph launches (the rebuild decision taken on the device in a
 * conditional node per step; graphs of 8 steps where possible, else one step per
 * graph); the host reads the device status once per
 * chunk of up to 200 steps.  If a rebuild inside a chunk outgrows the
 * list or tile capacity, the chunk is redone from a snapshot of its starting
 * state after the capacities have been regrown (md_info.n_redos counts these).
 * On the mixed-precision full-list path the force kernel of each step also
 * performs the velocity-Verlet updates around it (closing kick, and unless it
 * is the last step of the call, the next opening kick and drift): the same
 * operations as separate kernels, with the positions (FP32 and FP64)
 * double-buffered.  After md_set_tbsma the integration runs as separate kernels.
 * With the environment variable MDGB_NO_GRAPHS=1 set when the system is
 * created, the same kernels are launched from the host instead and the rebuild
 * flag is read after every step (slower; for profilers that do not follow
 * kernels into conditional graph nodes).  MDGB_NO_FUSE=1 at creation runs
 * force and integration as separate kernels (bit-identical results).
 * Energies are not computed on the way (use md_energy_virial).
 * Errors: MD_ERR_NONFINITE, MD_ERR_SKIN_VIOLATION, overflow codes, MD_ERR_CUDA.
 */
int md_step(md_system *s, int32_t n_steps);

/*
 * Potential energy, kinetic energy and virial W_ab = sum over pairs of
 * d_a f_b (d = x_i - x_j, f = force on i; components xx yy zz xy xz yz) at the
 * current state, reduced in FP64 in a fixed order (Sec. II.C thread-local
 * accumulators).  Any output pointer may be NULL.  Host outputs; synchronises.
 */
int md_energy_virial(md_system *s, double *pe, double *ke, double virial[6]);

/*
 * Replace the pair parameters (n_species x n_species row-major, symmetric; rcut
 * may be NULL for the r_cut given at creation).  No cutoff may exceed the
 * largest one the system was created with (the cell grid and list radius were
 * sized from it).  The neighbour lists stay valid; forces are recomputed on the
 * next call that needs them.  Host arrays.  Errors: MD_ERR_ARG.
 * No counterpart in the paper (the parameter-derivative functions below are
 * the force-matching extension).
 */
int md_set_params(md_system *s, const double *eps, const double *sigma, const double *rcut);

/*
 * Switch the system to the tight-binding second-moment many-body potential of
 * Cleri and Rosato (1993), the potential of all of the paper's benchmarks
 * (Sec. III; the paper gives no parameters):
 *   E = sum_i [ sum_j A exp(-p (r_ij/r0 - 1)) - sqrt( sum_j xi^2 exp(-2q (r_ij/r0 - 1)) ) ]
 * with both sums over the neighbours closer than r_cut (strict <; the pair set
 * is decided by the FP64 definition as for the pair potential).  Forces are
 * evaluated in two passes over the cell tasks (densities, then forces, which
 * need 1/sqrt(rho) of both atoms of a pair); md_forces, md_step and
 * md_energy_virial (per-atom energy sum_j phi - sqrt(rho)) use it until
 * md_set_params switches back to the pair table.  Units are the caller's (eV,
 * Angstrom and amu for the published copper set: A = 0.0855, xi = 1.224,
 * p = 10.960, q = 2.278, r0 = 2.5562).  md_step then runs velocity Verlet
 * with separate force and integration launches.  Requires one species,
 * MD_MIXED, MD_LIST_FULL, r_cut no larger than the cutoff the system was
 * created with (the lists' radius) and xi^2 exp(2q) < 2000 (the fixed-point
 * density range).  Errors: MD_ERR_ARG.  No derivatives (md_forces_backward)
 * for this potential.
 */
int md_set_tbsma(md_system *s, double A, double xi, double p, double q, double r0, double r_cut);

/*
 * Reverse-mode derivatives for force matching.  For a scalar loss L of the
 * forces at the current state, with grad_f = dL/dF (N x 3, original order)
 * given, writes
 *   grad_pos   dL/dx (N x 3, original order), NULL to skip;
 *   grad_eps   dL/deps, n_species x n_species, NULL to skip;
 *   grad_sigma dL/dsigma, likewise;
 * over the pairs inside their cutoffs, the pair set held fixed (the cutoff
 * contributes no derivative).  Per pair (i,j), d = x_i - x_j, f_ij = g d and
 * w = G_i - G_j: dL/dx_i += g w + 2 (dg/dr^2) (w.d) d and the negative on x_j;
 * dL/deps_ab += (w.d) g/eps; dL/dsig_ab += (w.d) dg/dsig.  The tables are
 * symmetric: entry [a][b] = [b][a] is the derivative with respect to the value
 * shared by the species pair {a,b}.  Arithmetic: FP64 on MD_FP64 systems;
 * FP32 pair terms (FP64 sums of the parameter terms) on MD_MIXED ones.  Needs
 * MD_LIST_FULL.  grad_f and grad_pos are device pointers when device_ptrs != 0;
 * the tables are host arrays.  Deterministic; synchronises.
 * Errors: MD_ERR_ARG (half lists, NULL grad_f), MD_ERR_STATE, MD_ERR_CUDA.
 */
int md_forces_backward(md_system *s, const double *grad_f, int device_ptrs, double *grad_pos,
                       double *grad_eps, double *grad_sigma);

/*
 * Derivatives of the potential energy with respect to the pair parameters at
 * the current state: dE/deps_ab = sum 4 (s6^2 - s6), dE/dsig_ab = sum
 * 24 eps (2 s6^2 - s6)/sig over the pairs inside their cutoffs (s6 =
 * (sig/r)^6); same table convention and arithmetic as md_forces_backward.
 * (dE/dx is minus the force, md_forces.)  Host outputs; synchronises.
 */
int md_energy_param_grad(md_system *s, double *de_deps, double *de_dsigma);

/*
 * Copy the state out in original order: positions as stored (unwrapped since
 * the last build; add image * L for fully unwrapped coordinates), velocities
 * and image counters (N x 3 int32).  Any output may be NULL.
 */
int md_get_state(md_system *s, double *pos, double *vel, int32_t *image, int device_ptrs);

/*
 * The neighbour pair set of the last build as unordered pairs (i, j), i < j,
 * original ids, sorted by (i, j).  *n_pairs receives the count; pairs (host,
 * 2 x n_pairs int32) may be NULL to query the count only.  Full lists list
 * each pair twice internally; it is reported once.  Synchronises.
 */
int md_get_neighbors(md_system *s, int64_t *n_pairs, int32_t *pairs);

/* Cell of every atom at the last binning (original order, linear index x fastest). Host output. */
int md_get_cells(md_system *s, int32_t *cell_of_atom);

/* Sizes and counters; host output. */
int md_get_info(md_system *s, md_info *out);

/*
 * Turn per-phase device timing on (enable != 0) or off.  While on, the
 * library brackets force evaluations and every binning + list build with CUDA
 * events on its stream and adds their elapsed times to md_info.force_ms and
 * md_info.build_ms; md_info.timed_force_evals and timed_builds count the
 * bracketed ones (the counters restart when timing is switched on).  In md_step's
 * 8-step graphs only the first step's force kernel is bracketed, so that the
 * events barely slow the steps they measure; every other force evaluation is.
 */
int md_set_timing(md_system *s, int enable);

/*
 * Race detector for the colour schedule of the half-list kernel (Sec. II.A: no
 * particle may be updated by two tasks of one wave; Sec. II.B).  On the GPU,
 * with the current binning, every 2x2x2-cell block of a phase tags each atom of
 * its 4x4x4-cell tile (the atoms its CTA writes) with its block id, by
 * compare-and-swap on a per-atom tag; an atom already tagged by another block
 * of the same phase is a conflict.  n_phases = 8 checks the 8 colour classes the
 * kernels use (conflicts must be 0); n_phases = 1 puts every block into one
 * phase, where overlapping tiles must show up.  *conflicts: the total over the
 * phases.  Debug use only (not on any timed path).  Errors: MD_ERR_ARG (n_phases
 * not 1 or 8, or n_phases = 8 on a full-list grid with a side of 4k+2 cells, which
 * has no colour classes), MD_ERR_STATE, MD_ERR_CUDA.
 */
int md_colour_conflicts(md_system *s, int32_t n_phases, int64_t *conflicts);

/*
 * Kinetic energy 1/2 sum m v^2 of n atoms, for callers that cannot allocate
 * device memory at the moment they need it - e.g. a host that gives this library
 * a fixed memory budget and locks allocation afterwards (an embedding runtime
 * that owns all device memory through its own pool), or a real-time loop that
 * must not call cudaMalloc, which can synchronise the device.
 * The paper has no counterpart of this call: it is a deployment variant of the
 * deterministic FP64 two-pass reduction md_energy_virial uses.  It needs no
 * md_system and allocates nothing: its partial sums live in a file-scope static
 * device array of 1024 doubles (8 KiB), which every GPU that loads the library
 * keeps until the process exits.
 *   vel      device, n x 3 doubles (any order); species: device, n int32, or NULL (all 0)
 *   mass     host, n_species doubles (1 <= n_species <= 4), copied by value
 *   ke_out   device, one double, written on `stream` (cudaStream_t, NULL = legacy default)
 * Every species id must lie in [0, n_species).  The ids are device data, so they
 * are checked on the device: an id outside that range contributes no mass and
 * makes *ke_out NaN (no memory outside mass[0 .. n_species) is read).
 * Limits and errors: MD_ERR_ARG if n < 0 or n > 2^30 (the largest size it
 * accepts), if ke_out or mass is NULL, or if n_species is out of range; nothing
 * is launched then.  MD_ERR_CUDA if a launch fails (the status of this call's
 * own launches; an error pending from earlier work is left as it is).
 * The first call on each device looks up the array's device address with that
 * device current (cudaGetSymbolAddress); make that first call before any stream
 * capture.  Every call overwrites the whole partial-sum array it uses, so nothing
 * has to start at zero, but all calls share the one array: calls whose kernels
 * overlap on the GPU (different streams, no ordering between them) race and may
 * return wrong sums.  Asynchronous: ke_out is valid once the stream reaches it.
 */
int md_kinetic_energy_noalloc(int64_t n, const double *vel, const int32_t *species,
                              const double *mass, int32_t n_species, double *ke_out, void *stream);

/* Copy the last error message into buf (at most len bytes, NUL-terminated). */
int md_last_error(md_system *s, char *buf, int64_t len);

/* Free all device workspace. NULL is allowed. */
void md_destroy(md_system *s);

#ifdef __cplusplus
}
#endif

#endif /* MDGB_H */
