/*
 * sc_oracle.c -- FP64 CPU oracle for Sutton-Chen Ni cluster molecular dynamics.
 *
 * TEST INFRASTRUCTURE. This file is the plain, slow, obviously-correct reference
 * that the CUDA path is checked against. Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it. The product library never
 * links, calls or falls back to it, and it shares no source with the CUDA path.
 *
 * Every quantity is IEEE double. Loops follow the definitions literally:
 *   - density            rho_i = sum_{j != i} (a / r_ij)^m                    (Eq. 2)
 *   - potential energy   U = eps * sum_i [ 1/2 sum_{j != i} (a/r_ij)^n
 *                                          - c * sqrt(rho_i) ]                 (Eq. 1)
 *   - force              F_i = -dU/dr_i, written out below (the paper prints no
 *                        force; the derivative of Eq. 1 is taken by hand)
 *   - the paper's two sweeps: first all rho_i, then the forces
 *                        (Sec. II, "Computational approach")
 *   - velocity-Verlet integration with a Langevin thermostat
 *                        (Sec. II, "Computational approach": Verlet integrator,
 *                        Langevin damping), in the BAOAB splitting.
 * Parallelism: an OpenMP loop over the outer atom index i only. The sum over j
 * for one i runs sequentially in index order inside one thread, so results do
 * not depend on the thread count.
 *
 * Readings of points the paper leaves open (units, mass, integrator splitting,
 * noise generator, ramp discretisation, Berendsen form, rho=0 guard, cutoff
 * form) are listed in the repository's design notes; each is restated where it
 * is used below.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- constants */
/* Unit system: Angstrom, femtosecond, atomic mass unit, electron-volt, kelvin.
 * (eV/amu) / (A/fs)^2 = e / u * 1e-10 with e = 1.602176634e-19 C (exact, SI 2019)
 * and u = 1.66053906660e-27 kg (CODATA 2018).                                */
#define ORC_EV_PER_AMU_A2_FS2 (1.602176634e-19 / 1.66053906660e-27 * 1.0e-10)
/* Boltzmann constant in eV/K (exact, SI 2019). */
#define ORC_KB_EV_PER_K 8.617333262e-5

typedef struct {
    double eps;   /* energy scale epsilon, eV            */
    double c;     /* dimensionless embedding weight c    */
    double a;     /* length scale a, Angstrom            */
    int n;        /* repulsive exponent n                */
    int m;        /* density exponent m                  */
    double rcut;  /* strict cutoff r < rcut in Angstrom; <= 0 means all pairs */
    int shift;    /* with a cutoff: 0 plain truncation; 1 every pair term inside rcut
                     shifted by its value at rcut, so the energy is continuous      */
    int reserved;
} orc_params;

typedef struct {
    int kind;          /* 0 = NVE, 1 = Langevin (BAOAB), 2 = Berendsen */
    double T0, T1;     /* linear ramp of the target temperature over the call, K */
    double gamma_ps;   /* Langevin friction, 1/ps */
    double tau_ps;     /* Berendsen coupling time, ps */
    uint64_t seed;     /* Philox key */
} orc_thermostat;

int orc_num_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

double orc_unit_ev_per_amu_a2_fs2(void) { return ORC_EV_PER_AMU_A2_FS2; }
double orc_unit_kb(void) { return ORC_KB_EV_PER_K; }

/* ------------------------------------------------------------------- pairs */
static double dist(const double* pos, int i, int j, double d[3]) {
    d[0] = pos[3 * i + 0] - pos[3 * j + 0];
    d[1] = pos[3 * i + 1] - pos[3 * j + 1];
    d[2] = pos[3 * i + 2] - pos[3 * j + 2];
    return sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
}

/* A pair interacts when j != i and, with a cutoff, when r < rcut strictly. */
static int interacts(double r, const orc_params* p) {
    return !(p->rcut > 0.0) || r < p->rcut;
}

/* The terms of one pair inside the cutoff: (a/r)^k, less (a/rcut)^k for the
 * shifted form, which then vanishes continuously at rcut. The shift does not
 * depend on r, so the derivatives (and the force formula below) are those of
 * the plain terms; only rho_i, and through it g_i, carry the shift.           */
static double term(double r, int k, const orc_params* p) {
    const double t = pow(p->a / r, k);
    return (p->shift && p->rcut > 0.0) ? t - pow(p->a / p->rcut, k) : t;
}

/* First sweep: rho_i = sum_{j != i} (a/r_ij)^m  (Eq. 2). */
void orc_density(int N, const double* pos, const orc_params* p, double* rho) {
    int i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < N; ++i) {
        double acc = 0.0, d[3];
        for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            double r = dist(pos, i, j, d);
            if (!interacts(r, p)) continue;
            acc += term(r, p->m, p);
        }
        rho[i] = acc;
    }
}

/* The embedding factor rho^(-1/2); defined as 0 when rho = 0 (an atom with no
 * partner in range), which is the limit of every term it multiplies.          */
static double inv_sqrt_rho(double rho) { return rho > 0.0 ? 1.0 / sqrt(rho) : 0.0; }

/*
 * Energy and forces of one isolated cluster.
 *   e_terms[0] = pair part      eps * 1/2 * sum_i sum_{j != i} (a/r_ij)^n
 *                (each term shifted by its value at rcut in the shifted form)
 *   e_terms[1] = embedding part -eps * c * sum_i sqrt(rho_i)
 * Force, from differentiating Eq. 1 (with s = a/r_ij, g_k = rho_k^(-1/2)):
 *   d(s^k)/dr = -k s^k / r and rho_j depends on r_i through the (i,j) term, so
 *   F_i = eps * sum_{j != i} [ n s^n - (c m / 2) (g_i + g_j) s^m ] (r_i - r_j) / r^2.
 * forces may be NULL; rho_out may be NULL.  Returns U = e_terms[0] + e_terms[1].
 */
double orc_energy_forces(int N, const double* pos, const orc_params* p, double* forces,
                         double* e_terms, double* rho_out) {
    double* rho = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    double* g = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    orc_density(N, pos, p, rho);
    for (int i = 0; i < N; ++i) g[i] = inv_sqrt_rho(rho[i]);

    /* Energy: per-atom pair sums (parallel over i), then plain sums in index order. */
    double* pair_i = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    {
        int i;
#pragma omp parallel for schedule(static)
        for (i = 0; i < N; ++i) {
            double acc = 0.0, d[3];
            for (int j = 0; j < N; ++j) {
                if (j == i) continue;
                double r = dist(pos, i, j, d);
                if (!interacts(r, p)) continue;
                acc += term(r, p->n, p);
            }
            pair_i[i] = acc;
        }
    }
    double e_pair = 0.0, e_emb = 0.0;
    for (int i = 0; i < N; ++i) {
        e_pair += 0.5 * p->eps * pair_i[i];
        e_emb += -p->eps * p->c * sqrt(rho[i]);
    }
    free(pair_i);

    if (forces) {
        int i;
        const double kemb = 0.5 * p->c * (double)p->m;
#pragma omp parallel for schedule(static)
        for (i = 0; i < N; ++i) {
            double f[3] = {0.0, 0.0, 0.0}, d[3];
            for (int j = 0; j < N; ++j) {
                if (j == i) continue;
                double r = dist(pos, i, j, d);
                if (!interacts(r, p)) continue;
                double s = p->a / r;
                double coef = p->eps * ((double)p->n * pow(s, p->n) -
                                        kemb * (g[i] + g[j]) * pow(s, p->m)) / (r * r);
                f[0] += coef * d[0];
                f[1] += coef * d[1];
                f[2] += coef * d[2];
            }
            forces[3 * i + 0] = f[0];
            forces[3 * i + 1] = f[1];
            forces[3 * i + 2] = f[2];
        }
    }
    if (e_terms) { e_terms[0] = e_pair; e_terms[1] = e_emb; }
    if (rho_out) memcpy(rho_out, rho, sizeof(double) * (size_t)N);
    free(rho);
    free(g);
    return e_pair + e_emb;
}

/* Per-atom energy eps_i = eps [1/2 sum_{j!=i} s^n - c sqrt(rho_i)] (the summand of Eq. 1). */
void orc_atom_energies(int N, const double* pos, const orc_params* p, double* e_atom) {
    double* rho = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    orc_density(N, pos, p, rho);
    int i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < N; ++i) {
        double acc = 0.0, d[3];
        for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            double r = dist(pos, i, j, d);
            if (!interacts(r, p)) continue;
            acc += term(r, p->n, p);
        }
        e_atom[i] = p->eps * (0.5 * acc - p->c * sqrt(rho[i]));
    }
    free(rho);
}

/* ------------------------------------------------------------ Philox 4x32-10 */
/* Counter-based generator of Salmon, Moraes, Dror and Shaw (SC'11): ten rounds of
 * two 32x32->64 multiplies with a Weyl-sequence key schedule.                  */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0, 1]: (k + 1) * 2^-32. */
static double u01(uint32_t k) { return ((double)k + 1.0) * (1.0 / 4294967296.0); }

/*
 * Three standard normals for one atom at one step: Philox key = (lo32(seed),
 * hi32(seed)), counter = (atom, cluster, lo32(step), hi32(step)); Box-Muller
 * (1958) on the word pairs (w0,w1) and (w2,w3); the fourth normal is unused.
 */
void orc_langevin_normals(uint64_t seed, uint32_t cluster, int64_t step, uint32_t atom,
                          double z[3]) {
    uint32_t ctr[4] = {atom, cluster, (uint32_t)((uint64_t)step & 0xffffffffu),
                       (uint32_t)((uint64_t)step >> 32)};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    const double two_pi = 6.283185307179586476925286766559;
    double r1 = sqrt(-2.0 * log(u01(w[0])));
    double r2 = sqrt(-2.0 * log(u01(w[2])));
    z[0] = r1 * cos(two_pi * u01(w[1]));
    z[1] = r1 * sin(two_pi * u01(w[1]));
    z[2] = r2 * cos(two_pi * u01(w[3]));
}

/* ------------------------------------------------------------- observables */
typedef struct {
    double epot, ekin, etot, T;
    double com[3], mom[3], angmom[3];
} orc_obs;

/* Kinetic energy 1/2 sum m v^2 in eV; temperature 2 E_kin / (3 N k_B). */
static double kinetic(int N, const double* vel, const double* mass) {
    double ke = 0.0;
    for (int i = 0; i < N; ++i)
        ke += 0.5 * mass[i] *
              (vel[3 * i] * vel[3 * i] + vel[3 * i + 1] * vel[3 * i + 1] + vel[3 * i + 2] * vel[3 * i + 2]);
    return ke / ORC_EV_PER_AMU_A2_FS2;
}

void orc_observables(int N, const double* pos, const double* vel, const double* mass,
                     const orc_params* p, orc_obs* o) {
    double e_terms[2];
    o->epot = N > 0 ? orc_energy_forces(N, pos, p, NULL, e_terms, NULL) : 0.0;
    o->ekin = kinetic(N, vel, mass);
    o->etot = o->epot + o->ekin;
    o->T = N > 0 ? 2.0 * o->ekin / (3.0 * N * ORC_KB_EV_PER_K) : 0.0;
    double M = 0.0;
    for (int k = 0; k < 3; ++k) { o->com[k] = 0.0; o->mom[k] = 0.0; o->angmom[k] = 0.0; }
    for (int i = 0; i < N; ++i) {
        M += mass[i];
        for (int k = 0; k < 3; ++k) {
            o->com[k] += mass[i] * pos[3 * i + k];
            o->mom[k] += mass[i] * vel[3 * i + k];
        }
    }
    for (int k = 0; k < 3; ++k) o->com[k] = M > 0.0 ? o->com[k] / M : 0.0;
    for (int i = 0; i < N; ++i) {
        double r[3] = {pos[3 * i] - o->com[0], pos[3 * i + 1] - o->com[1], pos[3 * i + 2] - o->com[2]};
        const double* v = vel + 3 * i;
        o->angmom[0] += mass[i] * (r[1] * v[2] - r[2] * v[1]);
        o->angmom[1] += mass[i] * (r[2] * v[0] - r[0] * v[2]);
        o->angmom[2] += mass[i] * (r[0] * v[1] - r[1] * v[0]);
    }
}

/* --------------------------------------------------------------- integrator */
/*
 * nsteps steps of one cluster from the state (pos, vel, forces = F(pos)).
 * dt in fs. step0 is the global step index of the first step (it keys the noise).
 * Target temperature of local step k (k = 0..nsteps-1): T0 + (T1 - T0) k / nsteps.
 *   NVE       : B A A B  (velocity Verlet)
 *   Langevin  : B A O A B with O exact: v <- c1 v + sqrt((1 - c1^2) kB T / m) xi,
 *               c1 = exp(-gamma dt)
 *   Berendsen : B A A B, then v <- lambda v with
 *               lambda = sqrt(1 + (dt / tau) (T_target / T_inst - 1)), T_inst from
 *               the velocities after the final B (lambda = 1 when T_inst = 0).
 * where B: v += dt/2 F/m, A: x += dt/2 v (NVE and Berendsen merge the two A's).
 */
int orc_md_cluster(int N, double* pos, double* vel, double* forces, const double* mass,
                   const orc_params* p, uint32_t cluster, int64_t step0, int64_t nsteps,
                   double dt, const orc_thermostat* th) {
    const double conv = ORC_EV_PER_AMU_A2_FS2;
    const double h = 0.5 * dt;
    for (int64_t k = 0; k < nsteps; ++k) {
        double T_target = th->T0 + (th->T1 - th->T0) * (double)k / (double)nsteps;
        for (int i = 0; i < N; ++i)
            for (int c = 0; c < 3; ++c) vel[3 * i + c] += h * forces[3 * i + c] * conv / mass[i];
        if (th->kind == 1) {
            double c1 = exp(-th->gamma_ps * 1.0e-3 * dt);
            for (int i = 0; i < N; ++i) {
                double z[3];
                orc_langevin_normals(th->seed, cluster, step0 + k, (uint32_t)i, z);
                double sigma = sqrt((1.0 - c1 * c1) * ORC_KB_EV_PER_K * T_target * conv / mass[i]);
                for (int c = 0; c < 3; ++c) {
                    pos[3 * i + c] += h * vel[3 * i + c];
                    vel[3 * i + c] = c1 * vel[3 * i + c] + sigma * z[c];
                    pos[3 * i + c] += h * vel[3 * i + c];
                }
            }
        } else {
            for (int i = 0; i < N; ++i)
                for (int c = 0; c < 3; ++c) pos[3 * i + c] += dt * vel[3 * i + c];
        }
        orc_energy_forces(N, pos, p, forces, NULL, NULL);
        for (int i = 0; i < N; ++i)
            for (int c = 0; c < 3; ++c) vel[3 * i + c] += h * forces[3 * i + c] * conv / mass[i];
        if (th->kind == 2 && N > 0) {
            double T_inst = 2.0 * kinetic(N, vel, mass) / (3.0 * N * ORC_KB_EV_PER_K);
            double lambda = T_inst > 0.0
                                ? sqrt(1.0 + (dt / (th->tau_ps * 1.0e3)) * (T_target / T_inst - 1.0))
                                : 1.0;
            for (int i = 0; i < 3 * N; ++i) vel[i] *= lambda;
        }
    }
    return 0;
}

/* A batch of independent clusters stored back to back (sizes[b] atoms each). */
int orc_md_batch(int n_clusters, const int32_t* sizes, double* pos, double* vel, double* forces,
                 const double* mass, const orc_params* p, int64_t step0, int64_t nsteps, double dt,
                 const orc_thermostat* th) {
    int64_t off = 0;
    for (int b = 0; b < n_clusters; ++b) {
        orc_md_cluster(sizes[b], pos + 3 * off, vel + 3 * off, forces + 3 * off, mass + off, p,
                       (uint32_t)b, step0, nsteps, dt, th);
        off += sizes[b];
    }
    return 0;
}
