/*
 * structure_oracle.c -- FP64 CPU oracle for the structural observables of one cluster.
 *
 * TEST INFRASTRUCTURE, on the same terms as sc_oracle.c: only the test-suite may
 * load it; the product library never links, calls or falls back to it, and the two
 * share no source.
 *
 * Plain definitions, written out as loops:
 *   - centre of mass      X = sum_i m_i x_i / sum_i m_i
 *   - radial distribution of the central atoms (Sec. III: the pair-distance
 *     histogram of the atoms near the cluster's centre): the core is the atoms
 *     with |x_i - X| < r_core; every ordered pair (c, j), c in the core and j any
 *     other atom of the cluster, counts once in bin floor(r_cj / bin) when that is
 *     below nbins
 *   - mean squared displacement from a reference configuration with the motion of
 *     the centre of mass removed (the diffusion estimate of Sec. III):
 *         MSD = (1/n) sum_sel |(x_i - X) - (x0_i - X0)|^2
 *     over the atoms with |x0_i - X0| < r_core at the reference (all atoms when
 *     r_core <= 0)
 *   - common-neighbour analysis (Honeycutt and Andersen, J. Phys. Chem. 91, 4950
 *     (1987)): two atoms are neighbours when r < r_nb. A bonded pair i-j gets the
 *     signature (k, b, l): k the common neighbours of i and j, b the bonds among
 *     those k atoms, l the bonds in the largest connected set of those b bonds.
 *     An atom with exactly 12 neighbours is fcc when all 12 signatures are 421,
 *     hcp when six are 421 and six 422, icosahedral when all 12 are 555; every
 *     other atom is "other".
 * Distances: dx = x_i - x_j per axis and r^2 = (dx*dx + dy*dy) + dz*dz, evaluated
 * as written (the oracle is compiled with -ffp-contract=off), r = sqrt(r^2).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORS_OTHER = 0, ORS_FCC = 1, ORS_HCP = 2, ORS_ICO = 3 };

static double r2_of(const double* pos, int i, int j) {
    const double dx = pos[3 * i] - pos[3 * j];
    const double dy = pos[3 * i + 1] - pos[3 * j + 1];
    const double dz = pos[3 * i + 2] - pos[3 * j + 2];
    return (dx * dx + dy * dy) + dz * dz;
}

void ors_com(int N, const double* pos, const double* mass, double X[3]) {
    double M = 0.0, s[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < N; ++i) {
        M += mass[i];
        for (int q = 0; q < 3; ++q) s[q] += mass[i] * pos[3 * i + q];
    }
    for (int q = 0; q < 3; ++q) X[q] = s[q] / M;
}

static double r_from(const double* pos, int i, const double X[3]) {
    const double dx = pos[3 * i] - X[0], dy = pos[3 * i + 1] - X[1], dz = pos[3 * i + 2] - X[2];
    return sqrt((dx * dx + dy * dy) + dz * dz);
}

/* counts[nbins] and *n_core are overwritten. */
void ors_rdf(int N, const double* pos, const double* mass, double r_core, double bin, int nbins, int64_t* counts,
             int* n_core) {
    double X[3];
    ors_com(N, pos, mass, X);
    memset(counts, 0, sizeof(int64_t) * (size_t)nbins);
    int nc = 0;
    for (int c = 0; c < N; ++c) {
        if (!(r_from(pos, c, X) < r_core)) continue;
        ++nc;
        for (int j = 0; j < N; ++j) {
            if (j == c) continue;
            const double r = sqrt(r2_of(pos, c, j));
            const double t = r / bin;
            if (t < (double)nbins) counts[(int)t] += 1;
        }
    }
    *n_core = nc;
}

double ors_msd(int N, const double* pos, const double* ref, const double* mass, double r_core, int* n_sel) {
    double X[3], X0[3];
    ors_com(N, pos, mass, X);
    ors_com(N, ref, mass, X0);
    double s = 0.0;
    int n = 0;
    for (int i = 0; i < N; ++i) {
        if (r_core > 0.0 && !(r_from(ref, i, X0) < r_core)) continue;
        double d2 = 0.0;
        for (int q = 0; q < 3; ++q) {
            const double d = (pos[3 * i + q] - X[q]) - (ref[3 * i + q] - X0[q]);
            d2 += d * d;
        }
        s += d2;
        ++n;
    }
    *n_sel = n;
    return n > 0 ? s / n : 0.0;
}

/* ---------------------------------------------------------------- CNA */
typedef struct {
    int* start; /* [N + 1] */
    int* list;  /* neighbours of i in ascending order: list[start[i] .. start[i+1]) */
} nblist;

static nblist neighbours(int N, const double* pos, double r_nb) {
    const double rn2 = r_nb * r_nb;
    nblist L;
    L.start = (int*)calloc((size_t)N + 1, sizeof(int));
    int* cnt = (int*)calloc((size_t)N, sizeof(int));
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            if (j != i && r2_of(pos, i, j) < rn2) ++cnt[i];
    for (int i = 0; i < N; ++i) L.start[i + 1] = L.start[i] + cnt[i];
    L.list = (int*)malloc(sizeof(int) * (size_t)(L.start[N] > 0 ? L.start[N] : 1));
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < N; ++i) {
        int k = L.start[i];
        for (int j = 0; j < N; ++j)
            if (j != i && r2_of(pos, i, j) < rn2) L.list[k++] = j;
    }
    free(cnt);
    return L;
}

static int is_neighbour(const nblist* L, int p, int q) {
    for (int k = L->start[p]; k < L->start[p + 1]; ++k)
        if (L->list[k] == q) return 1;
    return 0;
}

static int find_root(int* parent, int a) {
    while (parent[a] != a) a = parent[a];
    return a;
}

/* Signature (k, b, l) of the pair i-j (which need not be bonded). */
static void signature(const nblist* L, int i, int j, int out[3]) {
    int common[64];
    int k = 0;
    for (int a = L->start[i]; a < L->start[i + 1]; ++a) {
        const int p = L->list[a];
        if (p != j && is_neighbour(L, j, p) && k < 64) common[k++] = p;
    }
    /* bonds among the common neighbours, and the connected sets they form */
    int bond_a[64 * 63 / 2], bond_b[64 * 63 / 2];
    int b = 0;
    for (int x = 0; x < k; ++x)
        for (int y = x + 1; y < k; ++y)
            if (is_neighbour(L, common[x], common[y])) {
                bond_a[b] = x;
                bond_b[b] = y;
                ++b;
            }
    int parent[64];
    for (int x = 0; x < k; ++x) parent[x] = x;
    for (int e = 0; e < b; ++e) {
        const int ra = find_root(parent, bond_a[e]), rb = find_root(parent, bond_b[e]);
        if (ra != rb) parent[ra] = rb;
    }
    int per_set[64];
    memset(per_set, 0, sizeof(per_set));
    for (int e = 0; e < b; ++e) per_set[find_root(parent, bond_a[e])] += 1;
    int l = 0;
    for (int x = 0; x < k; ++x)
        if (per_set[x] > l) l = per_set[x];
    out[0] = k;
    out[1] = b;
    out[2] = l;
}

void ors_cna_signature(int N, const double* pos, double r_nb, int i, int j, int out[3]) {
    nblist L = neighbours(N, pos, r_nb);
    signature(&L, i, j, out);
    free(L.start);
    free(L.list);
}

/* cls[N]: ORS_OTHER / ORS_FCC / ORS_HCP / ORS_ICO; nnb[N] (may be NULL): neighbour counts. */
void ors_cna(int N, const double* pos, double r_nb, int* cls, int* nnb) {
    nblist L = neighbours(N, pos, r_nb);
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < N; ++i) {
        const int n = L.start[i + 1] - L.start[i];
        if (nnb) nnb[i] = n;
        cls[i] = ORS_OTHER;
        if (n != 12) continue;
        int n421 = 0, n422 = 0, n555 = 0;
        for (int a = L.start[i]; a < L.start[i + 1]; ++a) {
            int s[3];
            signature(&L, i, L.list[a], s);
            n421 += s[0] == 4 && s[1] == 2 && s[2] == 1;
            n422 += s[0] == 4 && s[1] == 2 && s[2] == 2;
            n555 += s[0] == 5 && s[1] == 5 && s[2] == 5;
        }
        if (n421 == 12)
            cls[i] = ORS_FCC;
        else if (n421 == 6 && n422 == 6)
            cls[i] = ORS_HCP;
        else if (n555 == 12)
            cls[i] = ORS_ICO;
    }
    free(L.start);
    free(L.list);
}
