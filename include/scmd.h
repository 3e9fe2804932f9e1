/*
 * scmd.h -- C ABI of libscmd: Sutton-Chen molecular dynamics of free nickel
 * clusters on one NVIDIA GB300 (sm_103a).
 *
 * What it computes (Yakubovich, Sushko, Schramm, Solov'yov, "Kinetics of
 * liquid-solid phase transition in large nickel clusters", arXiv:1210.3559):
 *   - the Sutton-Chen potential energy of an isolated cluster (Eq. 1)
 *       U = eps * sum_i [ 1/2 sum_{j!=i} (a/r_ij)^n - c * sqrt(rho_i) ],
 *   - with the local density (Eq. 2)  rho_i = sum_{j!=i} (a/r_ij)^m,
 *   - evaluated, as in the paper's GPU code, as two successive two-body sweeps:
 *     first every rho_i, then the forces (Sec. II, "Computational approach"),
 *   - the forces F_i = -dU/dr_i (not printed in the paper; derived from Eq. 1):
 *       F_i = eps sum_{j!=i} [ n s^n - (c m / 2)(rho_i^-1/2 + rho_j^-1/2) s^m ]
 *             (r_i - r_j) / r_ij^2,   s = a / r_ij,
 *   - velocity-Verlet integration with a Langevin thermostat (Sec. II,
 *     "Computational approach": Verlet integrator, Langevin damping), here in
 *     the BAOAB splitting, plus plain NVE and a Berendsen weak-coupling option,
 *     driven by a target temperature that ramps linearly within a call (the
 *     paper's heating/cooling ramps, Sec. III).
 *
 * Units: Angstrom, femtosecond, atomic mass unit, electron-volt, kelvin.
 * Arrays of 3-vectors are row-major [N][3] doubles (x0 y0 z0 x1 y1 z1 ...).
 * Several independent clusters ("batch") live in one context, stored back to
 * back: cluster b owns atoms off_b .. off_b + sizes[b] - 1, off_b = sum_{c<b} sizes[c].
 *
 * Conventions shared by every entry point:
 *   - Ownership: the caller owns every pointer it passes (host arrays, and the
 *     device arrays of the *_device calls); the library copies inputs and never
 *     keeps or frees a caller pointer after returning. A context's own device
 *     memory is allocated in stream order on the context's stream
 *     (cudaMallocAsync on md_config.stream, or on the stream the library creates)
 *     and freed by md_destroy.
 *   - Errors: every call returns an md_status and never aborts, prints or traps
 *     the GPU. After an error the context stays valid for md_last_error and
 *     md_destroy; MD_ERR_CUDA means a CUDA call failed (message in
 *     md_last_error) and the context should be destroyed.
 *   - Streams: all GPU work is ordered on one CUDA stream (md_config.stream, or
 *     a stream the library creates). Calls that return host data synchronise
 *     that stream; md_step does not return before its work has completed.
 *   - Threads: one context must not be used by two host threads at once.
 *   - No CPU fallback: without a usable sm_103a GPU every call that needs the
 *     GPU fails with MD_ERR_CUDA.
 */
#ifndef SCMD_H
#define SCMD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SCMD_ABI_VERSION 2

typedef enum {
    MD_OK = 0,
    MD_ERR_INVALID = 1,   /* bad argument (null pointer, size, non-finite input, ...) */
    MD_ERR_CUDA = 2,      /* a CUDA runtime call failed or no suitable GPU            */
    MD_ERR_OOM = 3,       /* device or host allocation failed                         */
    MD_ERR_NONFINITE = 4, /* a force, position or velocity became NaN/Inf on the GPU  */
    MD_ERR_TIMEOUT = 5,   /* a bounded device-side wait gave up (the all-pairs passes wait,
                             within a thread-block cluster, for the partial sums the other
                             CTAs push; a correct run never comes near the bound)       */
    MD_ERR_STATE = 6      /* call not valid in the context's current state            */
} md_status;

typedef enum {
    MD_PREC_FP64 = 0,  /* every pair term, sum and update in IEEE double                 */
    MD_PREC_MIXED = 1  /* FP32 pair terms and forces; FP64 rho, energies, x and v        */
} md_precision;

typedef enum {
    MD_PATH_AUTO = 0,     /* neighbour lists when rcut_A > 0 and the largest cluster has
                             >= 8192 atoms (or the cutoff is shifted); else all pairs, in
                             FP64 as MD_PATH_ALLPAIRS_HALF once the batch has >= 1216 of
                             its work units (about one 1100-atom cluster) and its clusters
                             are large (sum n^3 / sum n^2 >= 512 atoms)                  */
    MD_PATH_ALLPAIRS = 1, /* every ordered pair (with the cutoff test if rcut_A > 0)    */
    MD_PATH_CELLS = 2,    /* uniform cell grid of side >= rcut_A; requires rcut_A > 0    */
    MD_PATH_VERLET = 3,   /* neighbour lists of rcut_A + 1 A built on the cell grid, rebuilt
                             when an atom has moved 0.5 A; requires rcut_A > 0. FP64: per
                             atom, forces independent of the rebuild times. MIXED: the atoms
                             in reach of each quad of 4 nearby atoms, summed in list order, so a resumed run
                             (md_set_state) agrees to rounding rather than bit for bit      */
    MD_PATH_ALLPAIRS_HALF = 4 /* FP64 only: all pairs, each unordered pair evaluated once and
                             added to both atoms (Newton's third law), in work units of 32 x 16
                             atoms whose partial sums are added per atom in a fixed order
                             (deterministic; bitwise resume). MIXED: MD_ERR_INVALID         */
} md_path;

/* The cell path (not in the paper, which sums every pair and leaves cutoffs to
 * later work, Sec. II) gives each cluster a fixed cubic grid of G^3 cells of side
 * h >= rcut_A around its centre of mass at creation, with a margin beyond the
 * cluster's radius; atoms outside the grid are counted in its border cells, which
 * keeps the result exact. Each step bins the atoms (a cell holds at most 256;
 * md_create refuses an rcut_A whose cells would exceed that at the fcc density
 * 4 / a^3, and a step that overflows a cell returns MD_ERR_STATE) and sums each
 * atom over the 5 x 5 x 5 cell octants (side h/2) around its own. Pair terms, masks and the integrator are
 * those of the all-pairs path with the cutoff, so both agree to rounding order. */

/* Sutton-Chen parameters (Eq. 1, Eq. 2). Paper's Ni set (Sec. II A):
 * eps_eV = 1.5707e-2, a_A = 3.52, c = 39.432, n = 9, m = 6.
 * rcut_A <= 0: all pairs. rcut_A > 0: a pair enters both rho and the pair sum
 * only when r_ij < rcut_A. cutoff_shift = 0: plain truncation. cutoff_shift = 1
 * (needs rcut_A > 0; the cell and neighbour-list paths only): each pair inside
 * rcut_A contributes (a/r)^n - (a/rcut)^n to the pair sum and (a/r)^m -
 * (a/rcut)^m to rho, so the energy is continuous when pairs cross the cutoff;
 * forces are its gradient (the derivative formula of the plain terms, with the
 * shifted rho). Zero-initialise: reserved must be 0. */
typedef struct {
    double eps_eV;
    double c;
    double a_A;
    int32_t n;
    int32_t m;
    double rcut_A;
    int32_t cutoff_shift;
    int32_t reserved;
} md_sc_params;

/* Context configuration. Zero-initialise, then set what you need. */
typedef struct {
    int32_t precision;        /* md_precision                                              */
    int32_t path;             /* md_path                                                   */
    int32_t obs_every;        /* md_step records observables every this many steps; 0 = never */
    int32_t graph_chunk;      /* steps per captured CUDA graph; 0 = library default (256)  */
    int32_t tune;             /* 0: built-in launch table; 1: autotune at create time      */
    int32_t obs_capacity;     /* samples kept by md_obs_history (ring); 0 = 4096           */
    const char* tune_cache;   /* JSON file read/written by the autotuner; NULL = none      */
    uint64_t stream;          /* cudaStream_t to use; 0 = the library creates one          */
} md_config;

typedef enum { MD_NVE = 0, MD_LANGEVIN = 1, MD_BERENDSEN = 2 } md_thermo_kind;

/* Thermostat of one md_step call. The target temperature of local step
 * k = 0..nsteps-1 is T0_K + (T1_K - T0_K) * k / nsteps (a linear ramp; equal
 * values give a fixed temperature). Langevin: friction gamma_per_ps, Gaussian
 * noise from Philox4x32-10 keyed by seed with counter (atom, cluster, step).
 * Berendsen: coupling time tau_ps (> dt). NVE ignores every field but kind. */
typedef struct {
    int32_t kind;         /* md_thermo_kind */
    int32_t reserved;
    double T0_K;
    double T1_K;
    double gamma_per_ps;
    double tau_ps;
    uint64_t seed;
} md_thermostat;

/* Per-cluster observables. E_pot from Eq. 1; E_kin = 1/2 sum m v^2;
 * T = 2 E_kin / (3 N k_B); com = centre of mass; mom = sum m v (amu A/fs);
 * angmom = sum m (x - com) x v (amu A^2/fs). status: 0, or MD_ERR_NONFINITE. */
typedef struct {
    double epot_eV, ekin_eV, etot_eV, T_K;
    double com_A[3];
    double mom[3];
    double angmom[3];
    int64_t step;
    double time_fs;
    int32_t status;
    int32_t reserved;
} md_obs;

typedef struct md_ctx md_ctx;

/* ABI version compiled into the library (SCMD_ABI_VERSION). */
int32_t md_abi_version(void);

/*
 * Create a context holding n_clusters independent clusters.
 *   sizes[n_clusters]   atoms per cluster, each >= 1
 *   pos_A[Ntot][3]      positions (Angstrom), vel[Ntot][3] velocities (A/fs),
 *   mass_amu[Ntot]      masses (> 0), Ntot = sum(sizes)
 * vel_A_per_fs may be NULL (all zero). Every value must be finite. Computes the
 * forces of the initial state (velocity Verlet needs F at step 0) and sets the
 * step counter to 0. On success *out receives the context; on failure *out is
 * NULL and md_last_error(NULL) describes the error (per host thread).
 */
md_status md_create(const md_config* cfg, int32_t n_clusters, const int32_t* sizes,
                    const double* pos_A, const double* vel_A_per_fs, const double* mass_amu,
                    const md_sc_params* params, md_ctx** out);

/*
 * md_create from device memory the caller owns (for example PyTorch CUDA
 * tensors); the state is that of the MD runs of Sec. II ("Computational
 * approach") and Sec. III: positions, velocities and masses of every atom: pos_dev[Ntot][3], vel_dev[Ntot][3] (may be NULL: zero velocities)
 * and mass_dev[Ntot] are contiguous float64 arrays in the same layout as
 * md_create's, in device memory of the current device; sizes is a host array.
 * The work is ordered on cfg->stream, which must be the stream that produced
 * the arrays (or be synchronised with it). The arrays are only read, never kept
 * or freed. On the all-pairs path they are validated on the GPU (finite
 * positions and velocities, finite masses > 0; else MD_ERR_INVALID) and copied
 * into the context's layout by a kernel, with no host round trip. The cell and
 * neighbour-list paths size each cluster's grid from its positions on the host,
 * so there the three arrays are read back once first. Results are identical to
 * md_create with the same values. Errors as md_create.
 */
md_status md_create_device(const md_config* cfg, int32_t n_clusters, const int32_t* sizes,
                           const double* pos_dev, const double* vel_dev, const double* mass_dev,
                           const md_sc_params* params, md_ctx** out);

/*
 * Evaluate the potential energy and forces at the current positions with the
 * two passes (density, then forces). epot_eV[n_clusters] and
 * forces_eV_per_A[Ntot][3] are host arrays; either may be NULL.
 */
md_status md_energy_forces(md_ctx* ctx, double* epot_eV, double* forces_eV_per_A);

/* Densities rho_i (Eq. 2) of the last force evaluation, host array [Ntot]. */
md_status md_get_density(md_ctx* ctx, double* rho);

/*
 * Advance every cluster by nsteps steps of length dt_fs under thermostat th
 * (NULL = NVE). Work is issued as replays of captured CUDA graphs of
 * graph_chunk steps; the call returns after the last step completed. Returns
 * MD_ERR_NONFINITE if any force, position or velocity became non-finite (the
 * state is then undefined; restore a checkpoint with md_set_state).
 */
md_status md_step(md_ctx* ctx, int64_t nsteps, double dt_fs, const md_thermostat* th);

/* Observables of every cluster at the current state (one fresh force
 * evaluation). out[n_clusters]. */
md_status md_observables(md_ctx* ctx, md_obs* out);

/*
 * Observables recorded by md_step every obs_every steps, oldest first.
 * out receives up to max_samples samples of n_clusters records each
 * (out[s * n_clusters + b]); *n_samples receives the number written. Samples
 * older than obs_capacity are dropped. md_clear_history empties the ring.
 */
md_status md_obs_history(md_ctx* ctx, md_obs* out, int32_t max_samples, int32_t* n_samples);
md_status md_clear_history(md_ctx* ctx);

/* Checkpoint: copy positions, velocities (host [Ntot][3]) and the step counter
 * out of, or into, the context. md_set_state recomputes the forces. Because the
 * Langevin noise is a pure function of (seed, cluster, atom, step), resuming
 * from a checkpoint reproduces an uninterrupted run bit for bit on every path
 * but the MIXED neighbour lists, whose sums follow the list order of the last
 * rebuild; there it agrees to rounding (MD_PATH_CELLS is bitwise in MIXED). */
md_status md_get_state(md_ctx* ctx, double* pos_A, double* vel_A_per_fs, int64_t* step);
md_status md_set_state(md_ctx* ctx, const double* pos_A, const double* vel_A_per_fs, int64_t step);

/* The same checkpoint (positions and velocities of the Sec. II / III MD state)
 * through caller-owned device arrays [Ntot][3] (float64,
 * current device), converted to and from the context's layout by kernels on
 * the context's stream; both calls return after that work has completed.
 * md_get_state_device: either array may be NULL. md_set_state_device: both are
 * required; the values are validated on the GPU first (non-finite ->
 * MD_ERR_INVALID and the context is left unchanged), then the forces are
 * recomputed, as in md_set_state. */
md_status md_get_state_device(md_ctx* ctx, double* pos_dev, double* vel_dev, int64_t* step);
/* md_energy_forces into caller-owned device arrays: the potential energy of
 * every cluster (Eq. 1) into epot_dev[n_clusters] and the forces (the
 * derivative of Eq. 1) into forces_dev[Ntot][3], float64, current device;
 * either may be NULL. Same evaluation and values as md_energy_forces (MIXED
 * forces are FP32 values widened to FP64); returns after the copies are done. */
md_status md_energy_forces_device(md_ctx* ctx, double* epot_dev, double* forces_dev);
md_status md_set_state_device(md_ctx* ctx, const double* pos_dev, const double* vel_dev, int64_t step);

/* MIXED precision keeps pair coordinates in FP32 relative to one origin per
 * cluster, set to the cluster's centre of mass when the context is created and
 * kept fixed afterwards (so that forces depend on the positions alone and a
 * checkpoint restored into this context, or into one created from the same
 * initial positions, resumes bit for bit). md_recenter moves every origin to
 * the current centre of mass (useful after md_set_state with a configuration
 * far from the original one) and recomputes the forces. */
md_status md_recenter(md_ctx* ctx);

/* Forces of the current state as held by the context (host [Ntot][3]). */
md_status md_get_forces(md_ctx* ctx, double* forces_eV_per_A);

/*
 * Launch shape of the two pair passes: i-atoms per thread (ipt), warps per
 * CTA (warps) and CTAs per thread-block cluster (cluster). md_get_launch
 * reads the current choice; md_set_launch overrides it (values outside
 * ipt in {1,2} (or 4 for the density pass), warps in {2,4,8,16} with warps >= ipt,
 * cluster in 1..8 -> MD_ERR_INVALID).
 * which: 0 = density pass, 1 = force pass.
 */
md_status md_get_launch(const md_ctx* ctx, int32_t which, int32_t* ipt, int32_t* warps, int32_t* cluster);
md_status md_set_launch(md_ctx* ctx, int32_t which, int32_t ipt, int32_t warps, int32_t cluster);

/*
 * Autotuner: time every launch shape of both passes on the context's own
 * clusters (CUDA events, reps launches each) and keep the fastest (the cell
 * path has a single launch shape: nothing to tune, returns MD_OK). With
 * cfg.tune_cache set, results are stored in (and later read from) that JSON
 * file, keyed by GPU name, SM count, precision, path and workload shape.
 */
md_status md_autotune(md_ctx* ctx, int32_t reps);

/*
 * Mean device time (ms) of one launch of the density pass and of the force
 * pass: CUDA events on the context's stream around reps back-to-back launches
 * of one pass after warm-up (consecutive launches overlap through programmatic
 * dependent launch as inside a step; with the neighbour lists in FP64, each
 * pass includes its gather kernel). Pair-evaluation counts per launch are returned in *pairs
 * (ordered pairs visited per pass: sum N_b (N_b - 1) for all pairs; for the cell
 * path, every atom times the atoms of the 5 x 5 x 5 cell octants around its own,
 * self included, as binned at the current positions; for the MIXED lists, 4
 * per listed atom (one per atom of the quad) plus the 12 within each quad; for the FP64 lists, twice the
 * half-list entries). Any output
 * may be NULL.
 */
md_status md_time_passes(md_ctx* ctx, int32_t reps, double* ms_density, double* ms_force,
                         double* pairs);

/*
 * The FP32 lane-operation rate of the current device, measured (a property of
 * the hardware, not of the paper's method: the roofline denominator of the
 * pair sweeps of Eq. 1 and Eq. 2): every SM runs
 * independent FFMA chains (one FFMA = one lane operation) for reps timed
 * launches, *measured_ops_per_s = lane operations / CUDA-event time. Also
 * *derived_ops_per_s = SMs x 128 FP32 lanes x the maximum SM clock. This is
 * the denominator of the pair passes' roofline (they are FP32-pipe bound).
 * reps >= 1; MD_ERR_CUDA without a GPU.
 */
md_status md_fp32_peak(int32_t reps, double* measured_ops_per_s, double* derived_ops_per_s);

/* Number of GPU kernels issued per md_step step (all pairs: 2, or 4 with
 * MD_PATH_ALLPAIRS_HALF, cells: 5,
 * neighbour lists: 6 in MIXED, 13 in FP64, plus one Berendsen kernel, two with
 * cells or lists, and the observable kernels of recorded steps) and per graph
 * replay overhead (launches per chunk), for launch accounting. */
md_status md_launch_counts(const md_ctx* ctx, int32_t* per_step, int32_t* per_chunk);

/* The pair path the context runs (MD_PATH_ALLPAIRS, MD_PATH_CELLS or MD_PATH_VERLET;
 * MD_PATH_AUTO is resolved at create time) into *path. */
md_status md_get_path(const md_ctx* ctx, int32_t* path);

/* Last error message of ctx, or of the calling thread's last failed md_create when ctx is NULL. */
const char* md_last_error(const md_ctx* ctx);

/* Free the context and its device memory. NULL is ignored. */
void md_destroy(md_ctx* ctx);

/*
 * Philox4x32-10 (Salmon et al., SC'11) evaluated by the GPU kernel code the
 * Langevin thermostat uses: in[k*6 .. k*6+5] = (ctr0, ctr1, ctr2, ctr3, key0,
 * key1), out[k*4 .. k*4+3] = the four output words; host arrays, count >= 0.
 */
md_status md_philox4x32_10(const uint32_t* in, uint32_t* out, int32_t count);

/*
 * The Langevin thermostat's standard normals as the GPU computes them, for
 * atoms 0..n_atoms-1 of one cluster at one step (Box-Muller on Philox output,
 * counter (atom, cluster, step lo, step hi), key (seed lo, seed hi)).
 * precision selects the FP32 (MD_PREC_MIXED) or FP64 transform. out[n_atoms][3].
 */
md_status md_langevin_normals(uint64_t seed, uint32_t cluster, int64_t step, int32_t n_atoms,
                              int32_t precision, double* out);

/*
 * Energy and forces of one cluster with no device allocation. The paper has no
 * counterpart; this exists for callers that cannot allocate device memory, such
 * as a host framework whose own allocator owns all of the GPU's memory, or a
 * time-critical loop that must never enter the CUDA allocator.
 *   pos_dev[n_atoms][3]     positions (Angstrom), device memory, read only
 *   forces_dev[n_atoms][3]  forces (eV/A), device memory, written
 *   epot_dev[1]             total Sutton-Chen potential energy (eV), device memory, written
 *   stream                  cudaStream_t on which the work is queued (0 = default stream)
 * The caller owns all three buffers. The arithmetic is that of md_energy_forces
 * in MIXED precision (FP32 pair terms, FP64 rho and energy), all pairs, or the
 * strict cutoff when params->rcut_A > 0 (plain truncation: cutoff_shift must be
 * 0). The call queues its kernels and returns;
 * synchronise the stream before reading the outputs. Working data lives in one
 * fixed array compiled into the library (kept by every GPU that loads it until the
 * process exits), so n_atoms is limited to 1..16384: anything else returns
 * MD_ERR_INVALID with a message in md_last_error(NULL), as does a bad argument.
 * Every call on a device shares that array and it keeps the last call's contents:
 * calls whose work overlaps on the GPU (other streams, other host threads) race and
 * must be serialised by the caller. The first call on each device looks up the
 * array's device address (with that device current); make that first call before
 * starting any stream capture. That address belongs to the CUDA context current at
 * the first call: after cudaDeviceReset (or any teardown of the device's primary
 * context) the next call looks it up again, so that call too must come before any
 * capture. The outputs are not checked: coincident atoms or non-finite positions
 * give non-finite forces and energy while the call still returns MD_OK, so a
 * caller that may pass such input tests the outputs for finiteness itself.
 */
md_status md_energy_forces_noalloc(const double* pos_dev, int32_t n_atoms, const md_sc_params* params,
                                   double* forces_dev, double* epot_dev, uint64_t stream);

/* ------------------------------------------------------------------------
 * Structural observables (Sec. III), computed on the device from the current
 * positions; only the small results are copied back. Distances that decide a
 * bin or a neighbour are evaluated in FP64 as dx = x_i - x_j per axis,
 * r^2 = (dx dx + dy dy) + dz dz, r = sqrt(r^2), each step rounded once.
 * ------------------------------------------------------------------------ */

/* Pair-distance histogram of the central atoms of every cluster (the g(r) of
 * the atoms near the centre, Sec. III). The core of cluster b is its atoms
 * closer than r_core_A to its centre of mass; every ordered pair (c, j), c in
 * the core and j any other atom of b, adds one to counts[b][floor(r_cj / bin_A)]
 * when that is below nbins. counts[n_clusters][nbins] (host, overwritten);
 * n_core[n_clusters] (host, may be NULL). nbins in 1..8192, bin_A > 0,
 * r_core_A >= 0; else MD_ERR_INVALID. Accumulate frames on the host. */
md_status md_rdf(md_ctx* ctx, double r_core_A, double bin_A, int32_t nbins, int64_t* counts, int32_t* n_core);

/* Store the current positions as the reference of md_msd. The atoms averaged
 * are those closer than r_core_A to their cluster's centre of mass now (every
 * atom when r_core_A <= 0). */
md_status md_msd_reference(md_ctx* ctx, double r_core_A);

/* Mean squared displacement since the reference, with each cluster's
 * centre-of-mass motion removed: msd_A2[b] = mean over the selected atoms of
 * |(x_i - X) - (x0_i - X0)|^2 (X the centre of mass), in A^2; n_atoms[b] (may be
 * NULL) the atoms averaged. MD_ERR_STATE before any md_msd_reference. */
md_status md_msd(md_ctx* ctx, double* msd_A2, int32_t* n_atoms);

/* Common-neighbour analysis (Honeycutt and Andersen 1987; the crystalline
 * fraction of the cluster). Atoms closer than r_nb_A are neighbours; a bond i-j
 * has the signature (common neighbours, bonds among them, bonds in the largest
 * connected set of those). An atom with exactly 12 neighbours is fcc when all 12
 * signatures are 421, hcp when six are 421 and six 422, icosahedral when all are
 * 555; every other atom is "other". counts[n_clusters][4] (host): atoms that are
 * other, fcc, hcp, icosahedral. cls[Ntot] (host, may be NULL): 0..3 per atom.
 * capped[n_clusters] (host, may be NULL): atoms counted as other only because a
 * neighbour has more than 32 neighbours (none in a condensed metal at 3 A). */
md_status md_cna(md_ctx* ctx, double r_nb_A, int32_t* counts, int8_t* cls, int32_t* capped);

#ifdef __cplusplus
}
#endif
#endif /* SCMD_H */
