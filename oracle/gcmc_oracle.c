/*
 * gcmc_oracle.c -- plain, slow, FP64 CPU reference of the GCMC hot path of
 * "An Efficient Cell List Implementation for Monte Carlo Simulation on GPUs"
 * (Schwiebert, Hailat, Rushaidat, Mick, Potoff; arXiv 1408.3764).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header, table or
 * constant generator with the CUDA path.
 *
 * Everything here is written for clarity, not speed: plain loops, double
 * precision, no blocking, no fusion, no reordering beyond what the
 * definitions state.  Each function names the passage of the paper it
 * follows.
 *
 * Representation (a reading of the paper, which does not fix one):
 *   - cubic periodic box of edge L;
 *   - a particle coordinate is an unsigned 32-bit grid index X, its real
 *     position is x = X * h with h = L / 2^32 (positions live on a grid of
 *     spacing h, about 1e-8 sigma at the paper's box sizes);
 *   - the minimum-image separation of two particles along an axis is the
 *     signed grid difference wrapped into [-2^31, 2^31);
 *   - a pair is inside the cutoff iff the exact integer squared grid
 *     distance g is below R2 = ceil((rc * 2^32 / L)^2) (evaluated in IEEE
 *     double in exactly that order), i.e. r^2 < rc^2 decided exactly;
 *   - particle identity is (species s, index i), 0 <= i < N_s: species s
 *     owns its own dense index range, which is what a per-species
 *     deletion needs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_S 8
#define ORC_TWO32 4294967296.0

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: */
/* as easy as 1, 2, 3", SC'11).  Written from the published definition: */
/* ten rounds of two 32x32->64 multiplies with Weyl-sequence key bumps. */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------ */
/* Lennard-Jones pair energy, Eq. 1: U(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6]. */
/* Returns U and, through rep/att, the magnitudes of its two terms      */
/* (4 eps (sigma/r)^12 and 4 eps (sigma/r)^6), whose sum is the scale    */
/* of the rounding error of any evaluation of U.                        */
/* r2 == 0 (two particles on one grid point) is +inf by definition.      */
/* ------------------------------------------------------------------ */
double orc_lj(double r2, double eps, double sigma, double *rep, double *att)
{
    if (r2 == 0.0) {
        if (rep) *rep = INFINITY;
        if (att) *att = INFINITY;
        return INFINITY;
    }
    double r = sqrt(r2);
    double sr = sigma / r;
    double sr6 = sr * sr * sr * sr * sr * sr;
    double sr12 = sr6 * sr6;
    double a = 4.0 * eps * sr12;
    double b = 4.0 * eps * sr6;
    if (rep) *rep = a;
    if (att) *att = b;
    return a - b;
}

/* dU/dr of Eq. 1: 4 eps [-12 sigma^12 / r^13 + 6 sigma^6 / r^7]. */
double orc_lj_dr(double r2, double eps, double sigma)
{
    double r = sqrt(r2);
    double sr = sigma / r;
    double sr6 = sr * sr * sr * sr * sr * sr;
    return 4.0 * eps * (-12.0 * sr6 * sr6 + 6.0 * sr6) / r;
}

/* dU/dsigma of Eq. 1 at fixed r: 4 eps [12 sigma^11 / r^12 - 6 sigma^5 / r^6]. */
double orc_lj_dsigma(double r2, double eps, double sigma)
{
    double r = sqrt(r2);
    double sr = sigma / r;
    double sr6 = sr * sr * sr * sr * sr * sr;
    return 4.0 * eps * (12.0 * sr6 * sr6 - 6.0 * sr6) / sigma;
}

/* ------------------------------------------------------------------ */
/* System state                                                        */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t s;
    int32_t i;
} orc_ref;

typedef struct {
    double L, rc, h, q, V;
    int S;
    double eps[ORC_MAX_S * ORC_MAX_S];
    double sigma[ORC_MAX_S * ORC_MAX_S];
    int T;             /* cells per side (Sec. 3.2.2) */
    int64_t ncell;
    uint64_t R2;       /* cutoff on the squared grid distance */
    int64_t cap[ORC_MAX_S]; /* allocated indices per species (grows) */
    int64_t n[ORC_MAX_S];
    uint32_t *pos[ORC_MAX_S]; /* pos[s][3*i + axis] grid coordinates */
    /* cells: an ordered list of particle references per cell */
    int64_t *cell_len;
    int64_t *cell_alloc;
    orc_ref **cell;
    double E;          /* running total energy */
    double W;          /* running virial sum_{i<j} r U'(r) (NaN: not set) */
    /* microcells (Sec. 3.3): M per side, an ordered reference list per
     * microcell; mc_M = 0 while none are built */
    int mc_M;
    int64_t mc_ncell;
    int64_t *mc_len;
    int64_t *mc_alloc;
    orc_ref **mc;
} orc_sys;

/* Cells per side, Sec. 3.2.2: the largest T with S = L/T >= rc, and T = 3
 * (S = L/3) when L < 3 rc. */
int orc_cells_per_side(double L, double rc)
{
    double t = floor(L / rc);
    int T = (int)t;
    if (T < 3) T = 3;
    return T;
}

/* Grid quantisation of a real coordinate: X = floor(x * (2^32 / L)) mod 2^32.
 * Returns 0 on success, -1 when x is not finite or absurdly far outside. */
int orc_quantize(double x, double L, uint32_t *X)
{
    double q = ORC_TWO32 / L;
    double t = x * q;
    if (!(t == t) || t > 4.0e18 || t < -4.0e18) return -1;
    double f = floor(t);
    int64_t k = (int64_t)f;
    *X = (uint32_t)(uint64_t)k; /* modulo 2^32: periodic wrap */
    return 0;
}

/* The cutoff on the squared grid distance, as stated in the header. */
uint64_t orc_cutoff_grid2(double L, double rc)
{
    double q = ORC_TWO32 / L;
    double rq = rc * q;
    double rq2 = rq * rq;
    return (uint64_t)ceil(rq2);
}

/* Half-width of the displacement cube in grid units. */
int64_t orc_disp_grid(double max_disp, double L)
{
    double q = ORC_TWO32 / L;
    return (int64_t)(max_disp * q);
}

/* Cell coordinate of a grid coordinate: floor(x / S) = floor(X * T / 2^32). */
static int cell_coord(uint32_t X, int T)
{
    return (int)(((uint64_t)X * (uint64_t)T) >> 32);
}

static int64_t cell_of(const orc_sys *sys, const uint32_t P[3])
{
    int cx = cell_coord(P[0], sys->T);
    int cy = cell_coord(P[1], sys->T);
    int cz = cell_coord(P[2], sys->T);
    return ((int64_t)cz * sys->T + cy) * sys->T + cx;
}

/* Minimum-image grid separation along one axis: the difference wrapped
 * into [-2^31, 2^31) (Sec. 3.1, "true distance ... applying periodic
 * boundary conditions"). */
static int64_t min_image(uint32_t a, uint32_t b)
{
    int64_t d = (int64_t)a - (int64_t)b;
    if (d >= 2147483648LL) d -= 4294967296LL;
    if (d < -2147483648LL) d += 4294967296LL;
    return d;
}

orc_sys *orc_create(double L, double rc, int S, const double *eps, const double *sigma)
{
    if (!(L > 0.0) || !(rc > 0.0) || 2.0 * rc > L || S < 1 || S > ORC_MAX_S) return NULL;
    orc_sys *sys = (orc_sys *)calloc(1, sizeof(orc_sys));
    sys->L = L;
    sys->rc = rc;
    sys->h = L / ORC_TWO32;
    sys->q = ORC_TWO32 / L;
    sys->V = L * L * L;
    sys->S = S;
    for (int k = 0; k < S * S; ++k) {
        sys->eps[k] = eps[k];
        sys->sigma[k] = sigma[k];
    }
    sys->T = orc_cells_per_side(L, rc);
    sys->ncell = (int64_t)sys->T * sys->T * sys->T;
    sys->R2 = orc_cutoff_grid2(L, rc);
    for (int s = 0; s < S; ++s) {
        sys->cap[s] = 64;
        sys->pos[s] = (uint32_t *)calloc((size_t)(3 * sys->cap[s]), sizeof(uint32_t));
    }
    sys->cell_len = (int64_t *)calloc((size_t)sys->ncell, sizeof(int64_t));
    sys->cell_alloc = (int64_t *)calloc((size_t)sys->ncell, sizeof(int64_t));
    sys->cell = (orc_ref **)calloc((size_t)sys->ncell, sizeof(orc_ref *));
    return sys;
}

static void micro_free(orc_sys *sys)
{
    for (int64_t c = 0; c < sys->mc_ncell; ++c) free(sys->mc[c]);
    free(sys->mc);
    free(sys->mc_len);
    free(sys->mc_alloc);
    sys->mc = NULL;
    sys->mc_len = sys->mc_alloc = NULL;
    sys->mc_M = 0;
    sys->mc_ncell = 0;
}

void orc_destroy(orc_sys *sys)
{
    if (!sys) return;
    micro_free(sys);
    for (int s = 0; s < sys->S; ++s) free(sys->pos[s]);
    for (int64_t c = 0; c < sys->ncell; ++c) free(sys->cell[c]);
    free(sys->cell);
    free(sys->cell_len);
    free(sys->cell_alloc);
    free(sys);
}

int orc_geometry(const orc_sys *sys, int64_t *T, int64_t *ncell, uint64_t *R2, double *h)
{
    *T = sys->T;
    *ncell = sys->ncell;
    *R2 = sys->R2;
    *h = sys->h;
    return 0;
}

static void cell_append(orc_sys *sys, int64_t c, orc_ref r)
{
    if (sys->cell_len[c] == sys->cell_alloc[c]) {
        int64_t na = sys->cell_alloc[c] ? 2 * sys->cell_alloc[c] : 8;
        sys->cell[c] = (orc_ref *)realloc(sys->cell[c], (size_t)na * sizeof(orc_ref));
        sys->cell_alloc[c] = na;
    }
    sys->cell[c][sys->cell_len[c]++] = r;
}

/* Removal from a cell, Sec. 3.2.5: exhaustive search for the particle,
 * the last entry of the cell takes its place, the counter drops by one. */
static int cell_remove(orc_sys *sys, int64_t c, orc_ref r)
{
    int64_t n = sys->cell_len[c];
    for (int64_t k = 0; k < n; ++k) {
        if (sys->cell[c][k].s == r.s && sys->cell[c][k].i == r.i) {
            sys->cell[c][k] = sys->cell[c][n - 1];
            sys->cell_len[c] = n - 1;
            return 0;
        }
    }
    return -1;
}

/* Makes room for index i of species s. */
static void ensure_index(orc_sys *sys, int s, int64_t i)
{
    if (i < sys->cap[s]) return;
    int64_t nc = sys->cap[s];
    while (nc <= i) nc *= 2;
    sys->pos[s] = (uint32_t *)realloc(sys->pos[s], (size_t)(3 * nc) * sizeof(uint32_t));
    sys->cap[s] = nc;
}

/* ------------------------------------------------------------------ */
/* Microcells, Sec. 3.3: the box cut into M^3 cells of edge about one   */
/* sigma, each holding an ordered list of its particles.  Reading: M =  */
/* ceil(L / edge) cells per side of equal edge L / M (<= edge); the     */
/* paper's unit cells with a thinner last cell give the same counts of  */
/* cells per side.  The microcell of a grid coordinate X is             */
/* floor(X * M / 2^32), as for the ordinary cells.                      */
/* ------------------------------------------------------------------ */
static int64_t micro_of(const orc_sys *sys, const uint32_t P[3])
{
    int M = sys->mc_M;
    return ((int64_t)cell_coord(P[2], M) * M + cell_coord(P[1], M)) * M + cell_coord(P[0], M);
}

static void micro_append(orc_sys *sys, int64_t c, orc_ref r)
{
    if (sys->mc_len[c] == sys->mc_alloc[c]) {
        int64_t na = sys->mc_alloc[c] ? 2 * sys->mc_alloc[c] : 4;
        sys->mc[c] = (orc_ref *)realloc(sys->mc[c], (size_t)na * sizeof(orc_ref));
        sys->mc_alloc[c] = na;
    }
    sys->mc[c][sys->mc_len[c]++] = r;
}

/* Deleting an ID from a microcell, Sec. 3.3.3: scan the cell's list for it,
 * the last ID of the list takes its place, the counter drops by one. */
static int micro_remove(orc_sys *sys, int64_t c, orc_ref r)
{
    int64_t n = sys->mc_len[c];
    for (int64_t k = 0; k < n; ++k) {
        if (sys->mc[c][k].s == r.s && sys->mc[c][k].i == r.i) {
            sys->mc[c][k] = sys->mc[c][n - 1];
            sys->mc_len[c] = n - 1;
            return 0;
        }
    }
    return -1;
}

/* Builds the microcells of the current particles (Sec. 3.3.1): every
 * particle is added to the list of its microcell, species by species and
 * index by index.  Returns M, or -1 for a bad edge.  Later accepted moves
 * keep the lists up to date (orc_run_moves). */
int orc_micro_build(orc_sys *sys, double edge)
{
    if (!(edge > 0.0)) return -1;
    micro_free(sys);
    double m = ceil(sys->L / edge);
    if (m < 1.0) m = 1.0;
    if (m > 1024.0) return -1;
    sys->mc_M = (int)m;
    sys->mc_ncell = (int64_t)sys->mc_M * sys->mc_M * sys->mc_M;
    sys->mc_len = (int64_t *)calloc((size_t)sys->mc_ncell, sizeof(int64_t));
    sys->mc_alloc = (int64_t *)calloc((size_t)sys->mc_ncell, sizeof(int64_t));
    sys->mc = (orc_ref **)calloc((size_t)sys->mc_ncell, sizeof(orc_ref *));
    for (int s = 0; s < sys->S; ++s)
        for (int64_t i = 0; i < sys->n[s]; ++i) {
            orc_ref r = {s, (int32_t)i};
            micro_append(sys, micro_of(sys, &sys->pos[s][3 * i]), r);
        }
    return sys->mc_M;
}

/* Microcell state: per-cell counts and the concatenated per-cell lists
 * encoded as (i << 8) | s (either may be NULL); returns the largest count. */
int64_t orc_micro_state(const orc_sys *sys, int64_t *counts, uint32_t *refs)
{
    int64_t k = 0, mx = 0;
    for (int64_t c = 0; c < sys->mc_ncell; ++c) {
        if (counts) counts[c] = sys->mc_len[c];
        if (sys->mc_len[c] > mx) mx = sys->mc_len[c];
        if (refs)
            for (int64_t j = 0; j < sys->mc_len[c]; ++j)
                refs[k++] = ((uint32_t)sys->mc[c][j].i << 8) | (uint32_t)sys->mc[c][j].s;
    }
    return mx;
}

int orc_micro_per_side(const orc_sys *sys) { return sys->mc_M; }

static double pair_energy(const orc_sys *sys, const uint32_t A[3], int ta, const uint32_t B[3], int tb,
                          double *uabs);

/* The cube of microcells around microcell (cx, cy, cz), Sec. 3.3.2: thread
 * (tx, ty, tz) of an n x n x n cube, n = 2D + 1, takes the microcell at
 * offset (tx - D, ty - D, tz - D), wrapped around the periodic box.  When
 * n exceeds M the axis is taken whole, each cell once (offsets 0 .. M-1
 * from cell 0).  Writes the cells in thread order, x fastest; returns the
 * count (n_x n_y n_z). */
int64_t orc_micro_cube(const orc_sys *sys, int cx, int cy, int cz, int D, int64_t *cells)
{
    int M = sys->mc_M;
    int n = 2 * D + 1;
    int full = n > M;
    if (full) n = M;
    int64_t k = 0;
    for (int tz = 0; tz < n; ++tz)
        for (int ty = 0; ty < n; ++ty)
            for (int tx = 0; tx < n; ++tx) {
                int x = full ? tx : cx - D + tx;
                int y = full ? ty : cy - D + ty;
                int z = full ? tz : cz - D + tz;
                x = ((x % M) + M) % M;
                y = ((y % M) + M) % M;
                z = ((z % M) + M) % M;
                cells[k++] = ((int64_t)z * M + y) * M + x;
            }
    return k;
}

/* Energy of a particle of species t at P with every listed particle in the
 * cube of microcells (half-width D) around P's microcell, skipping particle
 * (excl_s, excl_i); adds |rep| + |att| to *uabs when given.  With a cube
 * that covers the cutoff this is the brute-force sum over all particles. */
double orc_energy_micro(const orc_sys *sys, const uint32_t P[3], int t, int excl_s, int64_t excl_i, int D,
                        double *uabs)
{
    int M = sys->mc_M;
    int64_t n = (int64_t)(2 * D + 1 < M ? 2 * D + 1 : M);
    int64_t *cells = (int64_t *)malloc((size_t)(n * n * n) * sizeof(int64_t));
    int64_t nc = orc_micro_cube(sys, cell_coord(P[0], M), cell_coord(P[1], M), cell_coord(P[2], M), D, cells);
    double e = 0.0;
    for (int64_t k = 0; k < nc; ++k) {
        int64_t c = cells[k];
        for (int64_t j = 0; j < sys->mc_len[c]; ++j) {
            orc_ref r = sys->mc[c][j];
            if (r.s == excl_s && r.i == excl_i) continue;
            e += pair_energy(sys, P, t, &sys->pos[r.s][3 * r.i], r.s, uabs);
        }
    }
    free(cells);
    return e;
}

/* Binning, Sec. 3.2.1.  Particles keep the order in which they are given:
 * the index of a particle within its species is its rank among the input
 * particles of that species, and every cell lists its particles in input
 * order (a stable counting sort by cell).  Also returns the compact cell
 * list: cell_start/cell_count per cell and order[] = input indices sorted
 * by cell (any of the three outputs may be NULL). */
int orc_build(orc_sys *sys, const double *pos, const int32_t *type, int64_t n,
              int64_t *cell_start, int64_t *cell_count, int64_t *order)
{
    for (int s = 0; s < sys->S; ++s) sys->n[s] = 0;
    for (int64_t c = 0; c < sys->ncell; ++c) sys->cell_len[c] = 0;
    micro_free(sys);
    int64_t *cellid = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    orc_ref *ref = (orc_ref *)malloc((size_t)(n > 0 ? n : 1) * sizeof(orc_ref));
    for (int64_t p = 0; p < n; ++p) {
        int s = type[p];
        if (s < 0 || s >= sys->S) {
            free(cellid);
            free(ref);
            return -1;
        }
        uint32_t P[3];
        for (int a = 0; a < 3; ++a)
            if (orc_quantize(pos[3 * p + a], sys->L, &P[a]) != 0) {
                free(cellid);
                free(ref);
                return -1;
            }
        int64_t i = sys->n[s]++;
        ensure_index(sys, s, i);
        for (int a = 0; a < 3; ++a) sys->pos[s][3 * i + a] = P[a];
        ref[p].s = s;
        ref[p].i = (int32_t)i;
        cellid[p] = cell_of(sys, P);
    }
    /* counting sort: histogram, exclusive prefix sum, stable placement */
    int64_t *cnt = (int64_t *)calloc((size_t)sys->ncell, sizeof(int64_t));
    for (int64_t p = 0; p < n; ++p) cnt[cellid[p]]++;
    int64_t *start = (int64_t *)calloc((size_t)sys->ncell, sizeof(int64_t));
    int64_t run = 0;
    for (int64_t c = 0; c < sys->ncell; ++c) {
        start[c] = run;
        run += cnt[c];
    }
    int64_t *fill = (int64_t *)calloc((size_t)sys->ncell, sizeof(int64_t));
    int64_t *ord = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t p = 0; p < n; ++p) {
        int64_t c = cellid[p];
        ord[start[c] + fill[c]++] = p;
    }
    for (int64_t c = 0; c < sys->ncell; ++c)
        for (int64_t k = 0; k < cnt[c]; ++k) cell_append(sys, c, ref[ord[start[c] + k]]);
    if (cell_start) memcpy(cell_start, start, (size_t)sys->ncell * sizeof(int64_t));
    if (cell_count) memcpy(cell_count, cnt, (size_t)sys->ncell * sizeof(int64_t));
    if (order) memcpy(order, ord, (size_t)n * sizeof(int64_t));
    free(cnt);
    free(start);
    free(fill);
    free(ord);
    free(cellid);
    free(ref);
    sys->E = NAN;
    sys->W = NAN;
    return 0;
}

/* Energy of one pair with exact cutoff decision; adds |rep|+|att| to *uabs,
 * |U| to *sabs when given (the scale of the per-move error measure
 * |dU_a - dU_b| / max(|dU|, 1e-3 sum_j |u_j|)) and, when wsum is given, the
 * pair's virial term r U'(r) to *wsum. */
static double pair_energy_w(const orc_sys *sys, const uint32_t A[3], int ta, const uint32_t B[3],
                            int tb, double *uabs, double *wsum, double *sabs)
{
    int64_t d[3];
    uint64_t g = 0;
    for (int a = 0; a < 3; ++a) {
        d[a] = min_image(A[a], B[a]);
        g += (uint64_t)(d[a] * d[a]);
    }
    if (g >= sys->R2) return 0.0;
    double dx = (double)d[0] * sys->h, dy = (double)d[1] * sys->h, dz = (double)d[2] * sys->h;
    double r2 = dx * dx + dy * dy + dz * dz;
    if (g == 0) r2 = 0.0;
    double rep, att;
    double u = orc_lj(r2, sys->eps[ta * sys->S + tb], sys->sigma[ta * sys->S + tb], &rep, &att);
    if (uabs) *uabs += rep + att;
    if (sabs) *sabs += fabs(u);
    if (wsum) *wsum += sqrt(r2) * orc_lj_dr(r2, sys->eps[ta * sys->S + tb], sys->sigma[ta * sys->S + tb]);
    return u;
}

static double pair_energy(const orc_sys *sys, const uint32_t A[3], int ta, const uint32_t B[3],
                          int tb, double *uabs)
{
    return pair_energy_w(sys, A, ta, B, tb, uabs, NULL, NULL);
}

/* Energy of a particle of species t at grid position P against every
 * particle of the system except (excl_s, excl_i) -- the definition the
 * energy decomposition evaluates (Algorithms 3 and 5: one thread per
 * particle, all particles, cutoff test). */
double orc_energy_brute(const orc_sys *sys, const uint32_t P[3], int t, int excl_s,
                        int64_t excl_i, double *uabs)
{
    double e = 0.0;
    if (uabs) *uabs = 0.0;
    for (int s = 0; s < sys->S; ++s)
        for (int64_t i = 0; i < sys->n[s]; ++i) {
            if (s == excl_s && i == excl_i) continue;
            e += pair_energy(sys, P, t, &sys->pos[s][3 * i], s, uabs);
        }
    return e;
}

/* The same energy restricted to the 27 cells around the cell of P
 * (Algorithms 6 and 7; Sec. 3.2: the home cell and its 26 neighbours).
 * T >= 3 makes the 27 cells distinct. */
static double energy_cells_w(const orc_sys *sys, const uint32_t P[3], int t, int excl_s,
                             int64_t excl_i, double *uabs, double *wsum, double *sabs)
{
    double e = 0.0;
    if (uabs) *uabs = 0.0;
    if (wsum) *wsum = 0.0;
    if (sabs) *sabs = 0.0;
    int T = sys->T;
    int cx = cell_coord(P[0], T), cy = cell_coord(P[1], T), cz = cell_coord(P[2], T);
    for (int oz = -1; oz <= 1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                int nx = (cx + ox + T) % T, ny = (cy + oy + T) % T, nz = (cz + oz + T) % T;
                int64_t c = ((int64_t)nz * T + ny) * T + nx;
                for (int64_t k = 0; k < sys->cell_len[c]; ++k) {
                    orc_ref r = sys->cell[c][k];
                    if (r.s == excl_s && r.i == excl_i) continue;
                    e += pair_energy_w(sys, P, t, &sys->pos[r.s][3 * r.i], r.s, uabs, wsum, sabs);
                }
            }
    return e;
}

double orc_energy_cells(const orc_sys *sys, const uint32_t P[3], int t, int excl_s,
                        int64_t excl_i, double *uabs)
{
    return energy_cells_w(sys, P, t, excl_s, excl_i, uabs, NULL, NULL);
}

/* Trial energies for m real positions (quantised by the grid rule).
 * exclude[k] = -1 for none, else (s << 32) | i.  brute != 0 uses the
 * all-particle sum instead of the 27 cells. */
int orc_trial_energy(const orc_sys *sys, const double *pos, const int32_t *species,
                     const int64_t *exclude, int64_t m, double *out, double *out_abs, int brute)
{
    for (int64_t k = 0; k < m; ++k) {
        uint32_t P[3];
        for (int a = 0; a < 3; ++a)
            if (orc_quantize(pos[3 * k + a], sys->L, &P[a]) != 0) return -1;
        int es = -1;
        int64_t ei = -1;
        if (exclude && exclude[k] >= 0) {
            es = (int)(exclude[k] >> 32);
            ei = exclude[k] & 0xffffffffLL;
        }
        double ua = 0.0;
        double e = brute ? orc_energy_brute(sys, P, species[k], es, ei, &ua)
                         : orc_energy_cells(sys, P, species[k], es, ei, &ua);
        out[k] = e;
        if (out_abs) out_abs[k] = ua;
    }
    return 0;
}

/* Total energy by its definition: the sum over unique pairs (Sec. 3.1.1). */
double orc_total_energy_brute(const orc_sys *sys)
{
    double e = 0.0;
    for (int s = 0; s < sys->S; ++s)
        for (int64_t i = 0; i < sys->n[s]; ++i)
            for (int s2 = s; s2 < sys->S; ++s2)
                for (int64_t j = (s2 == s ? i + 1 : 0); j < sys->n[s2]; ++j)
                    e += pair_energy(sys, &sys->pos[s][3 * i], s, &sys->pos[s2][3 * j], s2, NULL);
    return e;
}

/* Total energy through the cell list: half the sum of the per-particle
 * energies, each over its 27 cells. */
double orc_total_energy_cells(const orc_sys *sys)
{
    double e = 0.0;
    for (int s = 0; s < sys->S; ++s)
        for (int64_t i = 0; i < sys->n[s]; ++i)
            e += orc_energy_cells(sys, &sys->pos[s][3 * i], s, s, i, NULL);
    return 0.5 * e;
}

/* Per-particle energies e_i (species-major order). */
void orc_particle_energies(const orc_sys *sys, double *e)
{
    int64_t k = 0;
    for (int s = 0; s < sys->S; ++s)
        for (int64_t i = 0; i < sys->n[s]; ++i)
            e[k++] = orc_energy_cells(sys, &sys->pos[s][3 * i], s, s, i, NULL);
}

/* Analytic gradient of E = 1/2 sum_{i != j} U_{t_i t_j}(r_ij) (Eq. 1):
 *   dE/dr_i = sum_j U'(r) (r_i - r_j)/r            -> dpos (species-major, N x 3)
 *   dE/deps[a][b]   = 1/2 sum over ordered pairs of types (a,b) of U/eps
 *   dE/dsigma[a][b] = 1/2 sum over ordered pairs of types (a,b) of dU/dsigma
 *   virial = sum_{i<j} r U'(r)
 * Evaluated over the 27 cells of every particle; brute != 0 uses all pairs. */
int orc_energy_grad(const orc_sys *sys, double *dpos, double *deps, double *dsigma,
                    double *energy, double *virial, int brute)
{
    int S = sys->S, T = sys->T;
    double E = 0.0, W = 0.0;
    double ge[ORC_MAX_S * ORC_MAX_S], gs[ORC_MAX_S * ORC_MAX_S];
    for (int k = 0; k < S * S; ++k) ge[k] = gs[k] = 0.0;
    int64_t row = 0;
    for (int s = 0; s < S; ++s)
        for (int64_t i = 0; i < sys->n[s]; ++i, ++row) {
            const uint32_t *A = &sys->pos[s][3 * i];
            double f[3] = {0.0, 0.0, 0.0};
            /* visit every other particle j once: either all of them or
             * those of the 27 cells */
            int64_t ncand = 0;
            orc_ref *cand = NULL;
            if (brute) {
                int64_t tot = 0;
                for (int s2 = 0; s2 < S; ++s2) tot += sys->n[s2];
                cand = (orc_ref *)malloc((size_t)(tot > 0 ? tot : 1) * sizeof(orc_ref));
                for (int s2 = 0; s2 < S; ++s2)
                    for (int64_t j = 0; j < sys->n[s2]; ++j) {
                        cand[ncand].s = s2;
                        cand[ncand].i = (int32_t)j;
                        ++ncand;
                    }
            } else {
                int cx = cell_coord(A[0], T), cy = cell_coord(A[1], T), cz = cell_coord(A[2], T);
                int64_t tot = 0;
                for (int oz = -1; oz <= 1; ++oz)
                    for (int oy = -1; oy <= 1; ++oy)
                        for (int ox = -1; ox <= 1; ++ox) {
                            int64_t c = ((int64_t)((cz + oz + T) % T) * T + (cy + oy + T) % T) * T +
                                        (cx + ox + T) % T;
                            tot += sys->cell_len[c];
                        }
                cand = (orc_ref *)malloc((size_t)(tot > 0 ? tot : 1) * sizeof(orc_ref));
                for (int oz = -1; oz <= 1; ++oz)
                    for (int oy = -1; oy <= 1; ++oy)
                        for (int ox = -1; ox <= 1; ++ox) {
                            int64_t c = ((int64_t)((cz + oz + T) % T) * T + (cy + oy + T) % T) * T +
                                        (cx + ox + T) % T;
                            for (int64_t k = 0; k < sys->cell_len[c]; ++k) cand[ncand++] = sys->cell[c][k];
                        }
            }
            for (int64_t k = 0; k < ncand; ++k) {
                int s2 = cand[k].s;
                int64_t j = cand[k].i;
                if (s2 == s && j == i) continue;
                const uint32_t *B = &sys->pos[s2][3 * j];
                int64_t d[3];
                uint64_t g = 0;
                for (int a = 0; a < 3; ++a) {
                    d[a] = min_image(A[a], B[a]);
                    g += (uint64_t)(d[a] * d[a]);
                }
                if (g >= sys->R2) continue;
                double dx[3] = {(double)d[0] * sys->h, (double)d[1] * sys->h, (double)d[2] * sys->h};
                double r2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
                double e = sys->eps[s * S + s2], sg = sys->sigma[s * S + s2];
                double u = orc_lj(r2, e, sg, NULL, NULL);
                double du = orc_lj_dr(r2, e, sg);
                double r = sqrt(r2);
                for (int a = 0; a < 3; ++a) f[a] += du * dx[a] / r;
                E += 0.5 * u;
                W += 0.5 * r * du;
                ge[s * S + s2] += 0.5 * u / e;
                gs[s * S + s2] += 0.5 * orc_lj_dsigma(r2, e, sg);
            }
            free(cand);
            if (dpos)
                for (int a = 0; a < 3; ++a) dpos[3 * row + a] = f[a];
        }
    if (deps)
        for (int k = 0; k < S * S; ++k) deps[k] = ge[k];
    if (dsigma)
        for (int k = 0; k < S * S; ++k) dsigma[k] = gs[k];
    if (energy) *energy = E;
    if (virial) *virial = W;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Grand canonical Monte Carlo chain (Sec. 2, Algorithm 1)              */
/* ------------------------------------------------------------------ */
typedef struct {
    double p_disp, p_ins, p_del;
    double max_disp;
    double beta;
    double log_z[ORC_MAX_S]; /* ln z_s = beta mu_s - 3 ln Lambda */
} orc_mix;

typedef struct {
    double dU;      /* energy change of the trial */
    double lnA;     /* log of the acceptance ratio */
    double uabs;    /* sum over the evaluated pairs of |rep| + |att| */
    int32_t index;  /* particle index within its species (-1: none) */
    uint8_t type;   /* 0 displacement, 1 insertion, 2 deletion */
    uint8_t species;
    uint8_t accepted;
    uint8_t flagged;
} orc_trace;

typedef struct {
    int64_t attempted[3];
    int64_t accepted[3];
    int64_t flagged;
    int64_t moves_done;
    double energy;
    double sum_energy;
    double sum_n;
    int64_t n[ORC_MAX_S];
    double virial;      /* running virial after the last move */
    double sum_virial;  /* sum over the moves of the running virial */
} orc_stats;

void orc_set_energy(orc_sys *sys, double E) { sys->E = E; }
double orc_get_energy(const orc_sys *sys) { return sys->E; }
void orc_set_virial(orc_sys *sys, double W) { sys->W = W; }
double orc_get_virial(const orc_sys *sys) { return sys->W; }

/* The eight random words of move m of chain `chain`: two Philox blocks
 * with counter (m_lo, m_hi, chain, block) and key (seed_lo, seed_hi). */
void orc_move_words(uint64_t seed, uint64_t m, uint32_t chain, uint32_t w[8])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t c0[4] = {(uint32_t)m, (uint32_t)(m >> 32), chain, 0u};
    uint32_t c1[4] = {(uint32_t)m, (uint32_t)(m >> 32), chain, 1u};
    orc_philox4x32_10(c0, key, w);
    orc_philox4x32_10(c1, key, w + 4);
}

/* The particle a displacement (type 0) or a deletion (type 2) takes among
 * n >= 1 candidates.  Algorithm 1 takes one at random, uniformly; the paper
 * does not say how the index is drawn.  Reading: with 2^k the smallest power
 * of two that is at least n, the top k bits of independent words are tried
 * in turn and the first value below n is the index (rejection sampling, so
 * every index is equally likely).  A deletion tries w1, w2 and w3 (a
 * deletion does not use w2-w4 otherwise); a displacement tries w1 and, when
 * k <= 16, the top k bits of the low 16 bits of w1.  If no try is below n
 * the index is floor(f n / 2^32) of one more word f, independent of the
 * tries: w4 for a deletion, w5 for a displacement.  The index changes with
 * n only when n passes a power of two, when a try lies between the two
 * counts, or when every try fails. */
int64_t orc_pick_index(int64_t n, const uint32_t w[8], int type)
{
    int k = 0;
    while (((int64_t)1 << k) < n) ++k;
    if (k == 0) return 0; /* a single candidate */
    uint64_t tries[3];
    int ntries = 0;
    tries[ntries++] = (uint64_t)w[1] >> (32 - k);
    if (type == 2) {
        tries[ntries++] = (uint64_t)w[2] >> (32 - k);
        tries[ntries++] = (uint64_t)w[3] >> (32 - k);
    } else if (k <= 16) {
        tries[ntries++] = (uint64_t)(w[1] & 0xFFFFu) >> (16 - k);
    }
    for (int j = 0; j < ntries; ++j)
        if ((int64_t)tries[j] < n) return (int64_t)tries[j];
    uint32_t f = (type == 2) ? w[4] : w[5];
    return (int64_t)(((uint64_t)f * (uint64_t)n) >> 32);
}

/* Runs moves [first, first + n_moves) of the chain.  Per move (Algorithm 1
 * with the acceptance rules of Eqs. 3-5, read with the textbook sign of
 * the chemical potential):
 *   w0 picks the move type against thresholds floor(p * 2^32);
 *   displacement: particle k = orc_pick_index(N, w, 0) over all species in
 *     species-major order, each axis moves by ((w * (2D+1)) >> 32) - D grid
 *     units (D = the half-width in grid units), ln A = -beta dU;
 *   insertion: species (w5 * S) >> 32, grid position (w2, w3, w4),
 *     ln A = ln z_s + ln V - ln(N_s + 1) - beta dU;
 *   deletion: species (w5 * S) >> 32, index orc_pick_index(N_s, w, 2),
 *     ln A = ln N_s - ln z_s - ln V - beta dU (rejected when N_s = 0);
 *   u = ((w6 >> 5) * 2^26 + (w7 >> 6)) * 2^-53, accept iff ln u < ln A.
 * The cell list follows Sec. 3.2.5 (swap-with-last removal, append);
 * a deleted index is refilled by the last index of its species.
 * A trial is flagged when |ln u - ln A| <= beta * tol * uabs + 1e-12 * (1 + |ln A|).
 * Alongside the energy the chain keeps the virial W = sum_{i<j} r U'(r) (the
 * pair sum behind the virial pressure P = rho k T - W / (3V), Sec. 3.1.2):
 * each trial's dW is the same 27-cell sum with r U'(r) in place of U.
 * sum_abs_u (n_moves doubles, may be NULL) receives per move the sum of |u_j|
 * over the pair terms the trial evaluated (both positions of a displacement),
 * the floor of the per-move error measure |dU_a - dU_b| / max(|dU|, 1e-3
 * sum_j |u_j|) by which two evaluations of a trial are compared.
 * Returns 0, or -1 when the energy is not set. */
int orc_run_moves_ex(orc_sys *sys, uint64_t seed, uint32_t chain, uint64_t first, int64_t n_moves,
                     const orc_mix *mix, double tol, orc_trace *trace, orc_stats *st, double *sum_abs_u)
{
    memset(st, 0, sizeof(*st));
    if (!(sys->E == sys->E)) return -1;
    /* the running virial starts from the full sum over the 27 cells */
    if (!(sys->W == sys->W)) orc_energy_grad(sys, NULL, NULL, NULL, NULL, &sys->W, 0);
    int S = sys->S;
    uint64_t thr_disp = (uint64_t)(mix->p_disp * ORC_TWO32);
    uint64_t thr_ins = (uint64_t)((mix->p_disp + mix->p_ins) * ORC_TWO32);
    int64_t D = orc_disp_grid(mix->max_disp, sys->L);
    uint64_t span = (uint64_t)(2 * D + 1);
    double lnV = log(sys->V);
    for (int64_t mm = 0; mm < n_moves; ++mm) {
        uint64_t m = first + (uint64_t)mm;
        uint32_t w[8];
        orc_move_words(seed, m, chain, w);
        int type = (uint64_t)w[0] < thr_disp ? 0 : ((uint64_t)w[0] < thr_ins ? 1 : 2);
        uint64_t k53 = ((uint64_t)(w[6] >> 5) << 26) | (uint64_t)(w[7] >> 6);
        double u_acc = (double)k53 * (1.0 / 9007199254740992.0);
        double ln_u = log(u_acc);
        int64_t N = 0;
        for (int s = 0; s < S; ++s) N += sys->n[s];
        orc_trace tr;
        memset(&tr, 0, sizeof(tr));
        tr.type = (uint8_t)type;
        tr.index = -1;
        double dU = 0.0, lnA = -INFINITY, uabs = 0.0, dW = 0.0, sabs = 0.0;
        int s = 0;
        int64_t i = -1;
        int possible = 1;
        uint32_t Pn[3];
        if (type == 0) {
            if (N == 0) {
                possible = 0;
            } else {
                int64_t k = orc_pick_index(N, w, 0);
                s = 0;
                while (k >= sys->n[s]) {
                    k -= sys->n[s];
                    ++s;
                }
                i = k;
                const uint32_t *Po = &sys->pos[s][3 * i];
                for (int a = 0; a < 3; ++a) {
                    int64_t step = (int64_t)(((uint64_t)w[2 + a] * span) >> 32) - D;
                    Pn[a] = (uint32_t)((int64_t)Po[a] + step);
                }
                double ua0 = 0.0, ua1 = 0.0, w0 = 0.0, w1 = 0.0, sa0 = 0.0, sa1 = 0.0;
                double e_old = energy_cells_w(sys, Po, s, s, i, &ua0, &w0, &sa0);
                double e_new = energy_cells_w(sys, Pn, s, s, i, &ua1, &w1, &sa1);
                dU = e_new - e_old;
                dW = w1 - w0;
                uabs = ua0 + ua1;
                sabs = sa0 + sa1;
                lnA = -mix->beta * dU;
            }
        } else if (type == 1) {
            s = (int)(((uint64_t)w[5] * (uint64_t)S) >> 32);
            Pn[0] = w[2];
            Pn[1] = w[3];
            Pn[2] = w[4];
            dU = energy_cells_w(sys, Pn, s, -1, -1, &uabs, &dW, &sabs);
            i = sys->n[s];
            lnA = mix->log_z[s] + lnV - log((double)(sys->n[s] + 1)) - mix->beta * dU;
        } else {
            s = (int)(((uint64_t)w[5] * (uint64_t)S) >> 32);
            if (sys->n[s] == 0) {
                possible = 0;
            } else {
                i = orc_pick_index(sys->n[s], w, 2);
                double w0 = 0.0;
                dU = -energy_cells_w(sys, &sys->pos[s][3 * i], s, s, i, &uabs, &w0, &sabs);
                dW = -w0;
                lnA = log((double)sys->n[s]) - mix->log_z[s] - lnV - mix->beta * dU;
            }
        }
        int accept = 0, flag = 0;
        if (possible) {
            accept = ln_u < lnA;
            double band = mix->beta * tol * uabs + 1e-12 * (1.0 + fabs(lnA));
            flag = fabs(ln_u - lnA) <= band;
        }
        st->attempted[type]++;
        if (flag) st->flagged++;
        if (accept) {
            st->accepted[type]++;
            orc_ref r = {s, (int32_t)i};
            if (type == 0) {
                uint32_t *Po = &sys->pos[s][3 * i];
                int64_t c0 = cell_of(sys, Po), c1 = cell_of(sys, Pn);
                if (c0 != c1) {
                    cell_remove(sys, c0, r);
                    cell_append(sys, c1, r);
                }
                if (sys->mc_M) {
                    int64_t m0 = micro_of(sys, Po), m1 = micro_of(sys, Pn);
                    if (m0 != m1) {
                        micro_remove(sys, m0, r);
                        micro_append(sys, m1, r);
                    }
                }
                for (int a = 0; a < 3; ++a) Po[a] = Pn[a];
            } else if (type == 1) {
                ensure_index(sys, s, i);
                for (int a = 0; a < 3; ++a) sys->pos[s][3 * i + a] = Pn[a];
                sys->n[s]++;
                cell_append(sys, cell_of(sys, Pn), r);
                if (sys->mc_M) micro_append(sys, micro_of(sys, Pn), r);
            } else {
                uint32_t *Pd = &sys->pos[s][3 * i];
                cell_remove(sys, cell_of(sys, Pd), r);
                if (sys->mc_M) micro_remove(sys, micro_of(sys, Pd), r);
                int64_t last = sys->n[s] - 1;
                if (i != last) {
                    uint32_t *Pl = &sys->pos[s][3 * last];
                    int64_t cl = cell_of(sys, Pl);
                    for (int64_t k = 0; k < sys->cell_len[cl]; ++k)
                        if (sys->cell[cl][k].s == s && sys->cell[cl][k].i == last) sys->cell[cl][k].i = (int32_t)i;
                    if (sys->mc_M) {
                        int64_t ml = micro_of(sys, Pl);
                        for (int64_t k = 0; k < sys->mc_len[ml]; ++k)
                            if (sys->mc[ml][k].s == s && sys->mc[ml][k].i == last) sys->mc[ml][k].i = (int32_t)i;
                    }
                    for (int a = 0; a < 3; ++a) Pd[a] = Pl[a];
                }
                sys->n[s]--;
            }
            sys->E += dU;
            sys->W += dW;
        }
        if (trace) {
            tr.dU = dU;
            tr.lnA = lnA;
            tr.uabs = uabs;
            tr.index = (int32_t)i;
            tr.species = (uint8_t)s;
            tr.accepted = (uint8_t)accept;
            tr.flagged = (uint8_t)flag;
            trace[mm] = tr;
        }
        if (sum_abs_u) sum_abs_u[mm] = sabs;
        int64_t Nn = 0;
        for (int q = 0; q < S; ++q) Nn += sys->n[q];
        st->sum_energy += sys->E;
        st->sum_virial += sys->W;
        st->sum_n += (double)Nn;
        st->moves_done++;
    }
    st->energy = sys->E;
    st->virial = sys->W;
    for (int q = 0; q < S; ++q) st->n[q] = sys->n[q];
    return 0;
}

/* The chain without the per-move sums of |u_j|. */
int orc_run_moves(orc_sys *sys, uint64_t seed, uint32_t chain, uint64_t first, int64_t n_moves,
                  const orc_mix *mix, double tol, orc_trace *trace, orc_stats *st)
{
    return orc_run_moves_ex(sys, seed, chain, first, n_moves, mix, tol, trace, st, NULL);
}

/* Current state: particle counts per species, grid positions in
 * species-major order, per-cell counts and the concatenated per-cell
 * references encoded as (i << 8) | s. */
int64_t orc_count(const orc_sys *sys, int s) { return sys->n[s]; }

void orc_get_state(const orc_sys *sys, uint32_t *pos, int64_t *cell_count, uint32_t *cell_refs)
{
    int64_t row = 0;
    for (int s = 0; s < sys->S; ++s)
        for (int64_t i = 0; i < sys->n[s]; ++i, ++row)
            for (int a = 0; a < 3; ++a) pos[3 * row + a] = sys->pos[s][3 * i + a];
    int64_t k = 0;
    for (int64_t c = 0; c < sys->ncell; ++c) {
        if (cell_count) cell_count[c] = sys->cell_len[c];
        if (cell_refs)
            for (int64_t j = 0; j < sys->cell_len[c]; ++j)
                cell_refs[k++] = ((uint32_t)sys->cell[c][j].i << 8) | (uint32_t)sys->cell[c][j].s;
    }
}

/* Widom test-particle average <exp(-beta e(p))> over n random insertion
 * points of species t drawn from Philox with the given seed (used to pick
 * chemical potentials for the synthetic workloads). */
double orc_widom(const orc_sys *sys, int t, double beta, uint64_t seed, int64_t n)
{
    double acc = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        uint32_t w[4];
        uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
        uint32_t ctr[4] = {(uint32_t)k, (uint32_t)((uint64_t)k >> 32), 0xffffffffu, 7u};
        orc_philox4x32_10(ctr, key, w);
        uint32_t P[3] = {w[0], w[1], w[2]};
        double e = orc_energy_cells(sys, P, t, -1, -1, NULL);
        acc += exp(-beta * e);
    }
    return acc / (double)n;
}
