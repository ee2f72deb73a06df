/*
 * su3_oracle.c -- plain, slow FP64 CPU oracle of the checkerboard SU(3)
 * heatbath sweep (Berg & Wu, "Fortran MPI Checkerboard Code for SU(3) Lattice
 * Gauge Theory II", arXiv:0904.1179).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline / reference arm may load this library.  The CUDA
 * library never links, includes or calls it, and this file uses nothing from
 * the CUDA side.
 *
 * What the paper fixes (and what this file follows):
 *   - pure SU(3) lattice gauge theory with the Wilson action, Markov chain
 *     Monte Carlo, periodic boundary conditions (Sec. 1, Introduction);
 *   - checkerboard updating: links of one direction and one site parity are
 *     updated together (Abstract; Sec. 1; Appendix A, Eq. (mscb18) counts the
 *     checkerboard half-lattice storage mscb);
 *   - the MPI code uses a "1-hit" heatbath update of each SU(3) matrix
 *     (Sec. 2.1, remark on the non-MPI program's repeat-until-accepted
 *     heatbath and the 97.2% 1-hit acceptance at beta = 5.7);
 *   - PBC through neighbour pointer arrays, the common implementation that
 *     Sec. 2.1 mentions in its paragraph on the boundary exchange cost;
 *   - one timed unit = one SU(3) matrix update (Sec. 2.1, Fig. 1 caption);
 *   - start-configuration creation is separate from the sweeps (Sec. 2).
 * Everything else is silent in the paper and follows these textbook
 * readings: Wilson action S = beta sum_P (1 - ReTr U_P / 3),
 * Cabibbo-Marinari (Phys. Lett. B119 (1982) 387) over the SU(2) subgroups
 * (0,1), (0,2), (1,2), Kennedy-Pendleton (Phys. Lett. B156 (1985) 393)
 * sampling with one hit, Gram-Schmidt reunitarisation after every update,
 * and Philox4x32-10 (Salmon et al., SC'11) as the counter-based generator.
 *
 * Host layout (canonical): double U[L3][L2][L1][L0][4 mu][3 row][3 col][2 re/im],
 * site index s = x0 + L0*(x1 + L1*(x2 + L2*x3)), parity p = (x0+x1+x2+x3) mod 2.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, so
 * every product and sum is rounded exactly as written).
 *
 * Parity pinning: every exported function is pinned by a CPU test against
 * something other than itself (known-answer vectors, closed forms, invariants,
 * strong/weak-coupling limits, brute force); see tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 4.2): 10 rounds,   */
/* each round two 32x32->64 multiplications and a key-dependent xor, with a  */
/* Weyl-sequence key bump between rounds.                                    */
/* ------------------------------------------------------------------------ */
static const uint32_t PHILOX_MULT_A = 0xD2511F53u;
static const uint32_t PHILOX_MULT_B = 0xCD9E8D57u;
static const uint32_t PHILOX_WEYL_A = 0x9E3779B9u; /* golden ratio */
static const uint32_t PHILOX_WEYL_B = 0xBB67AE85u; /* sqrt(3) - 1 */

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    int round;
    for (round = 0; round < 10; round++) {
        uint64_t prod_a, prod_b;
        uint32_t n0, n1, n2, n3;
        if (round > 0) {
            k0 += PHILOX_WEYL_A;
            k1 += PHILOX_WEYL_B;
        }
        prod_a = (uint64_t)PHILOX_MULT_A * (uint64_t)c0;
        prod_b = (uint64_t)PHILOX_MULT_B * (uint64_t)c2;
        n0 = (uint32_t)(prod_b >> 32) ^ c1 ^ k0;
        n1 = (uint32_t)prod_b;
        n2 = (uint32_t)(prod_a >> 32) ^ c3 ^ k1;
        n3 = (uint32_t)prod_a;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0,1) from two 32-bit words: 52 bits (a<<20 | b>>12), centred in
 * its bin, so the result lies in [2^-53, 1 - 2^-53] and is exact. */
double oracle_u01_f64(uint32_t a, uint32_t b)
{
    uint64_t x = ((uint64_t)a << 20) | (uint64_t)(b >> 12);
    return ((double)x + 0.5) * 2.220446049250313080847263336181640625e-16; /* 2^-52 */
}

/* Uniform in (0,1) from one word for the FP32-mixed reading: 23 bits. */
double oracle_u01_f32(uint32_t a)
{
    uint32_t x = a >> 9;
    return ((double)x + 0.5) * 1.1920928955078125e-07; /* 2^-23 */
}

/* Counter layout: (site, mu | sub<<2 | call<<4, sweep low word,
 * tag | (sweep high word)<<4); key = (seed low, seed high).
 * tag 0 = link update, 1 = hot start, 2 = gauge transformation, 3 = sampler test. */
static void draw_words(uint64_t seed, uint32_t site, uint32_t w1, uint64_t t, uint32_t tag, uint32_t out[4])
{
    uint32_t ctr[4], key[2];
    ctr[0] = site;
    ctr[1] = w1;
    ctr[2] = (uint32_t)t;
    ctr[3] = tag | ((uint32_t)(t >> 32) << 4);
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32);
    oracle_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* 3x3 complex matrices, written out element by element.                    */
/* ------------------------------------------------------------------------ */
typedef struct { double re, im; } cplx;
typedef struct { cplx e[3][3]; } mat3;

static cplx c_mul(cplx a, cplx b) { cplx r; r.re = a.re * b.re - a.im * b.im; r.im = a.re * b.im + a.im * b.re; return r; }
static cplx c_conj(cplx a) { cplx r; r.re = a.re; r.im = -a.im; return r; }
static cplx c_add(cplx a, cplx b) { cplx r; r.re = a.re + b.re; r.im = a.im + b.im; return r; }
static cplx c_sub(cplx a, cplx b) { cplx r; r.re = a.re - b.re; r.im = a.im - b.im; return r; }
static cplx c_scale(cplx a, double s) { cplx r; r.re = a.re * s; r.im = a.im * s; return r; }

static mat3 m_mul(const mat3* a, const mat3* b)
{
    mat3 r;
    int i, j, k;
    for (i = 0; i < 3; i++)
        for (j = 0; j < 3; j++) {
            cplx s = {0.0, 0.0};
            for (k = 0; k < 3; k++) s = c_add(s, c_mul(a->e[i][k], b->e[k][j]));
            r.e[i][j] = s;
        }
    return r;
}

static mat3 m_dag(const mat3* a)
{
    mat3 r;
    int i, j;
    for (i = 0; i < 3; i++)
        for (j = 0; j < 3; j++) r.e[i][j] = c_conj(a->e[j][i]);
    return r;
}

static mat3 m_zero(void)
{
    mat3 r;
    memset(&r, 0, sizeof r);
    return r;
}

static void m_acc(mat3* a, const mat3* b)
{
    int i, j;
    for (i = 0; i < 3; i++)
        for (j = 0; j < 3; j++) a->e[i][j] = c_add(a->e[i][j], b->e[i][j]);
}

static double re_trace(const mat3* a) { return a->e[0][0].re + a->e[1][1].re + a->e[2][2].re; }

/* Third row of an SU(3) matrix from its first two: conj(row0 x row1). */
static void third_row(mat3* u)
{
    cplx a = c_sub(c_mul(u->e[0][1], u->e[1][2]), c_mul(u->e[0][2], u->e[1][1]));
    cplx b = c_sub(c_mul(u->e[0][2], u->e[1][0]), c_mul(u->e[0][0], u->e[1][2]));
    cplx c = c_sub(c_mul(u->e[0][0], u->e[1][1]), c_mul(u->e[0][1], u->e[1][0]));
    u->e[2][0] = c_conj(a);
    u->e[2][1] = c_conj(b);
    u->e[2][2] = c_conj(c);
}

/* Gram-Schmidt on rows 0 and 1, then row 2 = conj(row0 x row1). */
static void reunitarise(mat3* u)
{
    double n0 = 0.0, n1 = 0.0;
    cplx d = {0.0, 0.0};
    int k;
    for (k = 0; k < 3; k++) n0 += u->e[0][k].re * u->e[0][k].re + u->e[0][k].im * u->e[0][k].im;
    n0 = 1.0 / sqrt(n0);
    for (k = 0; k < 3; k++) u->e[0][k] = c_scale(u->e[0][k], n0);
    for (k = 0; k < 3; k++) d = c_add(d, c_mul(c_conj(u->e[0][k]), u->e[1][k]));
    for (k = 0; k < 3; k++) u->e[1][k] = c_sub(u->e[1][k], c_mul(d, u->e[0][k]));
    for (k = 0; k < 3; k++) n1 += u->e[1][k].re * u->e[1][k].re + u->e[1][k].im * u->e[1][k].im;
    n1 = 1.0 / sqrt(n1);
    for (k = 0; k < 3; k++) u->e[1][k] = c_scale(u->e[1][k], n1);
    third_row(u);
}

/* ------------------------------------------------------------------------ */
/* Lattice geometry: canonical index and neighbour pointer tables.          */
/* ------------------------------------------------------------------------ */
typedef struct {
    int L[4];
    int64_t V;
    int64_t* up; /* up[s*4+nu] = s + nu-hat */
    int64_t* dn; /* dn[s*4+nu] = s - nu-hat */
} geom;

static void site_coords(const int L[4], int64_t s, int x[4])
{
    x[0] = (int)(s % L[0]); s /= L[0];
    x[1] = (int)(s % L[1]); s /= L[1];
    x[2] = (int)(s % L[2]); s /= L[2];
    x[3] = (int)s;
}

static int64_t site_index(const int L[4], const int x[4])
{
    return (int64_t)x[0] + (int64_t)L[0] * ((int64_t)x[1] + (int64_t)L[1] * ((int64_t)x[2] + (int64_t)L[2] * (int64_t)x[3]));
}

static int site_parity(const int L[4], int64_t s)
{
    int x[4];
    site_coords(L, s, x);
    return (x[0] + x[1] + x[2] + x[3]) & 1;
}

static int geom_init(geom* g, const int L[4])
{
    int64_t s;
    int nu;
    memcpy(g->L, L, sizeof g->L);
    g->V = (int64_t)L[0] * L[1] * L[2] * L[3];
    g->up = (int64_t*)malloc(sizeof(int64_t) * 4 * (size_t)g->V);
    g->dn = (int64_t*)malloc(sizeof(int64_t) * 4 * (size_t)g->V);
    if (!g->up || !g->dn) {
        free(g->up); free(g->dn);
        return -2;
    }
    for (s = 0; s < g->V; s++) {
        int x[4], y[4];
        site_coords(L, s, x);
        for (nu = 0; nu < 4; nu++) {
            memcpy(y, x, sizeof y);
            y[nu] = (x[nu] + 1) % L[nu];
            g->up[s * 4 + nu] = site_index(L, y);
            y[nu] = (x[nu] + L[nu] - 1) % L[nu];
            g->dn[s * 4 + nu] = site_index(L, y);
        }
    }
    return 0;
}

static void geom_free(geom* g)
{
    free(g->up);
    free(g->dn);
}

static int check_dims(const int L[4])
{
    int mu;
    for (mu = 0; mu < 4; mu++)
        if (L[mu] < 2 || (L[mu] & 1)) return -1;
    return 0;
}

/* Link access in the canonical layout. With f32 storage rows 0 and 1 are the
 * stored (float-representable) numbers and row 2 is rebuilt from them. */
static mat3 load_link(const double* U, int64_t s, int mu, int f32)
{
    mat3 m;
    const double* p = U + ((size_t)s * 4 + (size_t)mu) * 18;
    int i, j;
    for (i = 0; i < 3; i++)
        for (j = 0; j < 3; j++) {
            m.e[i][j].re = p[(i * 3 + j) * 2];
            m.e[i][j].im = p[(i * 3 + j) * 2 + 1];
        }
    if (f32) third_row(&m);
    return m;
}

static void store_link(double* U, int64_t s, int mu, mat3 m, int f32)
{
    double* p = U + ((size_t)s * 4 + (size_t)mu) * 18;
    int i, j;
    if (f32) {
        for (i = 0; i < 2; i++)
            for (j = 0; j < 3; j++) {
                m.e[i][j].re = (double)(float)m.e[i][j].re;
                m.e[i][j].im = (double)(float)m.e[i][j].im;
            }
        third_row(&m);
    }
    for (i = 0; i < 3; i++)
        for (j = 0; j < 3; j++) {
            p[(i * 3 + j) * 2] = m.e[i][j].re;
            p[(i * 3 + j) * 2 + 1] = m.e[i][j].im;
        }
}

/* ------------------------------------------------------------------------ */
/* Staple: the sum over nu != mu of the two three-link paths that close a    */
/* plaquette with U_mu(x), so that the link's share of the Wilson action is */
/* -(beta/3) Re Tr(U_mu(x) A).                                               */
/*   A = sum_nu  U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+                            */
/*             + U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu)                      */
/* ------------------------------------------------------------------------ */
static mat3 staple(const geom* g, const double* U, int64_t s, int mu, int f32)
{
    mat3 A = m_zero();
    int nu;
    int64_t s_pmu = g->up[s * 4 + mu];
    for (nu = 0; nu < 4; nu++) {
        int64_t s_pnu, s_mnu, s_pmu_mnu;
        mat3 a, b, c, t1, t2, t3;
        if (nu == mu) continue;
        s_pnu = g->up[s * 4 + nu];
        s_mnu = g->dn[s * 4 + nu];
        s_pmu_mnu = g->dn[s_pmu * 4 + nu];
        /* forward (upper) staple */
        a = load_link(U, s_pmu, nu, f32);
        b = load_link(U, s_pnu, mu, f32);
        c = load_link(U, s, nu, f32);
        t1 = m_dag(&b);
        t2 = m_mul(&a, &t1);
        t1 = m_dag(&c);
        t3 = m_mul(&t2, &t1);
        m_acc(&A, &t3);
        /* backward (lower) staple */
        a = load_link(U, s_pmu_mnu, nu, f32);
        b = load_link(U, s_mnu, mu, f32);
        c = load_link(U, s_mnu, nu, f32);
        t1 = m_dag(&a);
        t2 = m_dag(&b);
        t3 = m_mul(&t1, &t2);
        t1 = m_mul(&t3, &c);
        m_acc(&A, &t1);
    }
    return A;
}

/* ------------------------------------------------------------------------ */
/* Kennedy-Pendleton one-hit SU(2) heatbath for the weight                    */
/*   P(a) da  ~  exp(alpha a0) dHaar(a),  i.e.  sqrt(1-a0^2) exp(alpha a0) da0 */
/* from six uniforms u[0..5]. Returns 1 and fills a[0..3] if accepted.        */
/* ------------------------------------------------------------------------ */
static int kp_one_hit(double alpha, const double u[6], double a[4])
{
    double c = cos(2.0 * ORACLE_PI * u[1]);
    double delta = -(log(u[0]) + c * c * log(u[2])) / alpha;
    double a0, rho, ct, st, phi;
    if (u[3] * u[3] > 1.0 - 0.5 * delta) return 0;
    a0 = 1.0 - delta;
    rho = 1.0 - a0 * a0;
    rho = rho > 0.0 ? sqrt(rho) : 0.0;
    ct = 1.0 - 2.0 * u[4];
    st = 1.0 - ct * ct;
    st = st > 0.0 ? sqrt(st) : 0.0;
    phi = 2.0 * ORACLE_PI * u[5];
    a[0] = a0;
    a[1] = rho * st * cos(phi);
    a[2] = rho * st * sin(phi);
    a[3] = rho * ct;
    return 1;
}

/* Six uniforms of proposal `tr` (0 for the one-hit heatbath) of subgroup
 * `sub` of the update of link (s, mu) at sweep t. */
static void subgroup_uniforms(uint64_t seed, int64_t s, int mu, int sub, int tr, uint64_t t, int f32, double u[6])
{
    uint32_t w[4];
    const uint32_t base = (uint32_t)(mu | (sub << 2)) | ((uint32_t)tr << 6);
    if (!f32) {
        int call;
        for (call = 0; call < 3; call++) {
            draw_words(seed, (uint32_t)s, base | (uint32_t)(call << 4), t, 0u, w);
            u[2 * call] = oracle_u01_f64(w[0], w[1]);
            u[2 * call + 1] = oracle_u01_f64(w[2], w[3]);
        }
    } else {
        draw_words(seed, (uint32_t)s, base, t, 0u, w);
        u[0] = oracle_u01_f32(w[0]);
        u[1] = oracle_u01_f32(w[1]);
        u[2] = oracle_u01_f32(w[2]);
        u[3] = oracle_u01_f32(w[3]);
        draw_words(seed, (uint32_t)s, base | (1u << 4), t, 0u, w);
        u[4] = oracle_u01_f32(w[0]);
        u[5] = oracle_u01_f32(w[1]);
    }
}

/* SU(2) element (quaternion a) as the 2x2 matrix [[a0+i a3, a2+i a1], [-a2+i a1, a0-i a3]]. */
static void su2_from_quaternion(const double a[4], cplx m[2][2])
{
    m[0][0].re = a[0];  m[0][0].im = a[3];
    m[0][1].re = a[2];  m[0][1].im = a[1];
    m[1][0].re = -a[2]; m[1][0].im = a[1];
    m[1][1].re = a[0];  m[1][1].im = -a[3];
}

/* One Cabibbo-Marinari update of link (s, mu): three SU(2) subgroups, each
 * a Kennedy-Pendleton heatbath in the field of the staple A, then GS.
 * max_tries = 1 is the one-hit heatbath of the MPI code; max_tries > 1
 * repeats the proposal until it is accepted, at most max_tries times (the
 * non-MPI program's repeat-until-accepted heatbath, Sec. 2.1 remark).
 * stats[0] counts accepted proposals, stats[1] proposals drawn (a degenerate
 * subgroup counts as one). */
static mat3 update_link(const geom* g, const double* U, double beta, uint64_t seed, uint64_t t, int64_t s, int mu,
                        int f32, int max_tries, uint64_t* stats, double* margins)
{
    static const int sub_rows[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    mat3 A = staple(g, U, s, mu, f32);
    mat3 u = load_link(U, s, mu, f32);
    int sub;
    for (sub = 0; sub < 3; sub++) {
        int i = sub_rows[sub][0], j = sub_rows[sub][1];
        mat3 W = m_mul(&u, &A);
        double r[4], k, uu[6], a[4];
        int tr;
        r[0] = 0.5 * (W.e[i][i].re + W.e[j][j].re);
        r[1] = 0.5 * (W.e[i][j].im + W.e[j][i].im);
        r[2] = 0.5 * (W.e[i][j].re - W.e[j][i].re);
        r[3] = 0.5 * (W.e[i][i].im - W.e[j][j].im);
        k = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3]);
        if (margins) margins[sub] = NAN;
        if (!(k > 1e-300)) { /* degenerate staple: measure zero, leave the subgroup */
            if (stats) stats[1]++;
            continue;
        }
        for (tr = 0; tr < max_tries; tr++) {
            subgroup_uniforms(seed, s, mu, sub, tr, t, f32, uu);
            if (stats) stats[1]++;
            if (margins && tr == 0) {
                /* distance of the first proposal's accept test from its threshold */
                double c = cos(2.0 * ORACLE_PI * uu[1]);
                double delta = -(log(uu[0]) + c * c * log(uu[2])) / (2.0 * beta * k / 3.0);
                margins[sub] = uu[3] * uu[3] - (1.0 - 0.5 * delta);
            }
            if (kp_one_hit(2.0 * beta * k / 3.0, uu, a)) {
                cplx y[2][2], v[2][2], vd[2][2], R[2][2];
                double rn[4];
                int p, q, col;
                rn[0] = r[0] / k; rn[1] = r[1] / k; rn[2] = r[2] / k; rn[3] = r[3] / k;
                su2_from_quaternion(a, y);
                su2_from_quaternion(rn, v);
                for (p = 0; p < 2; p++)
                    for (q = 0; q < 2; q++) vd[p][q] = c_conj(v[q][p]);
                for (p = 0; p < 2; p++)
                    for (q = 0; q < 2; q++) R[p][q] = c_add(c_mul(y[p][0], vd[0][q]), c_mul(y[p][1], vd[1][q]));
                for (col = 0; col < 3; col++) {
                    cplx ui = u.e[i][col], uj = u.e[j][col];
                    u.e[i][col] = c_add(c_mul(R[0][0], ui), c_mul(R[0][1], uj));
                    u.e[j][col] = c_add(c_mul(R[1][0], ui), c_mul(R[1][1], uj));
                }
                if (stats) stats[0]++;
                break;
            }
        }
    }
    reunitarise(&u);
    return u;
}

/* ------------------------------------------------------------------------ */
/* Exported entry points. Return 0 on success, -1 bad argument, -2 no memory. */
/* ------------------------------------------------------------------------ */

int oracle_cold_start(const int L[4], double* U)
{
    int64_t V, n, s;
    int mu;
    if (check_dims(L)) return -1;
    V = (int64_t)L[0] * L[1] * L[2] * L[3];
    n = V * 4 * 18;
    memset(U, 0, sizeof(double) * (size_t)n);
    for (s = 0; s < V; s++)
        for (mu = 0; mu < 4; mu++) {
            double* p = U + ((size_t)s * 4 + (size_t)mu) * 18;
            p[0] = 1.0; p[8] = 1.0; p[16] = 1.0;
        }
    return 0;
}

/* Haar-random SU(3) from two complex Gaussian rows (Box-Muller on Philox
 * words with tag `tag`), Gram-Schmidt and the completing third row. */
static mat3 haar_su3(uint64_t seed, int64_t s, int mu, uint32_t tag)
{
    mat3 m;
    double gz[12];
    int call, k;
    for (call = 0; call < 6; call++) {
        uint32_t w[4];
        double ua, ub, rad;
        draw_words(seed, (uint32_t)s, (uint32_t)(mu | (call << 4)), 0u, tag, w);
        ua = oracle_u01_f64(w[0], w[1]);
        ub = oracle_u01_f64(w[2], w[3]);
        rad = sqrt(-2.0 * log(ua));
        gz[2 * call] = rad * cos(2.0 * ORACLE_PI * ub);
        gz[2 * call + 1] = rad * sin(2.0 * ORACLE_PI * ub);
    }
    for (k = 0; k < 3; k++) {
        m.e[0][k].re = gz[2 * k];
        m.e[0][k].im = gz[2 * k + 1];
        m.e[1][k].re = gz[6 + 2 * k];
        m.e[1][k].im = gz[6 + 2 * k + 1];
    }
    reunitarise(&m);
    return m;
}

int oracle_hot_start(const int L[4], uint64_t seed, int f32, double* U)
{
    int64_t V, s;
    int mu;
    if (check_dims(L)) return -1;
    V = (int64_t)L[0] * L[1] * L[2] * L[3];
    for (s = 0; s < V; s++)
        for (mu = 0; mu < 4; mu++) store_link(U, s, mu, haar_su3(seed, s, mu, 1u), f32);
    return 0;
}

/* Mean plaquette (1/(6V)) sum_x sum_{mu<nu} (1/3) Re Tr U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+. */
double oracle_plaquette(const int L[4], const double* U, int f32)
{
    geom g;
    int64_t s;
    double sum = 0.0;
    if (check_dims(L)) return NAN;
    if (geom_init(&g, L)) return NAN;
    for (s = 0; s < g.V; s++) {
        int mu, nu;
        for (mu = 0; mu < 4; mu++)
            for (nu = mu + 1; nu < 4; nu++) {
                mat3 a = load_link(U, s, mu, f32);
                mat3 b = load_link(U, g.up[s * 4 + mu], nu, f32);
                mat3 c = load_link(U, g.up[s * 4 + nu], mu, f32);
                mat3 d = load_link(U, s, nu, f32);
                mat3 cd = m_dag(&c), dd = m_dag(&d);
                mat3 t1 = m_mul(&a, &b);
                mat3 t2 = m_mul(&t1, &cd);
                mat3 t3 = m_mul(&t2, &dd);
                sum += re_trace(&t3) / 3.0;
            }
    }
    geom_free(&g);
    return sum / (6.0 * (double)g.V);
}

/* Staple of link (site, mu), written as 18 doubles (row, col, re/im). */
int oracle_staple(const int L[4], const double* U, int64_t site, int mu, int f32, double* out)
{
    geom g;
    mat3 A;
    int i, j;
    if (check_dims(L) || mu < 0 || mu > 3) return -1;
    if (geom_init(&g, L)) return -2;
    if (site < 0 || site >= g.V) { geom_free(&g); return -1; }
    A = staple(&g, U, site, mu, f32);
    for (i = 0; i < 3; i++)
        for (j = 0; j < 3; j++) {
            out[(i * 3 + j) * 2] = A.e[i][j].re;
            out[(i * 3 + j) * 2 + 1] = A.e[i][j].im;
        }
    geom_free(&g);
    return 0;
}

/* One checkerboard half-sweep: every link U_mu(x) with parity(x) == parity is
 * updated once at sweep index t.  `reverse` walks the sites backwards (the
 * result must not depend on it).  stats[0] += accepted, stats[1] += proposed
 * SU(2) hits (stats may be NULL). */
int oracle_half_sweep(const int L[4], double beta, uint64_t seed, uint64_t t, int mu, int parity, int f32, int reverse,
                      double* U, uint64_t* stats, int max_tries)
{
    geom g;
    int64_t i;
    if (check_dims(L) || mu < 0 || mu > 3 || parity < 0 || parity > 1 || !(beta > 0.0) || !isfinite(beta)) return -1;
    if (max_tries < 1) return -1;
    if (geom_init(&g, L)) return -2;
    for (i = 0; i < g.V; i++) {
        int64_t s = reverse ? g.V - 1 - i : i;
        if (site_parity(L, s) != parity) continue;
        store_link(U, s, mu, update_link(&g, U, beta, seed, t, s, mu, f32, max_tries, stats, NULL), f32);
    }
    geom_free(&g);
    return 0;
}

/* nsweeps full sweeps starting at sweep index t0; a sweep is mu = 0..3, and
 * for each mu the even then the odd sites.  plaq (may be NULL) receives the
 * mean plaquette after each sweep. */
int oracle_sweep(const int L[4], double beta, uint64_t seed, uint64_t t0, int nsweeps, int f32, double* U, uint64_t* stats,
                 double* plaq, int max_tries)
{
    int n, mu, p, rc;
    for (n = 0; n < nsweeps; n++) {
        for (mu = 0; mu < 4; mu++)
            for (p = 0; p < 2; p++) {
                rc = oracle_half_sweep(L, beta, seed, t0 + (uint64_t)n, mu, p, f32, 0, U, stats, max_tries);
                if (rc) return rc;
            }
        if (plaq) plaq[n] = oracle_plaquette(L, U, f32);
    }
    return 0;
}

/* Update only the listed links (all of direction mu, at sweep index t), in
 * list order, in place.  Used for sampled checks on large lattices and for the
 * single-link equilibrium test. */
int oracle_update_links(const int L[4], double beta, uint64_t seed, uint64_t t, int mu, const int64_t* sites, int64_t n,
                        int f32, double* U, uint64_t* stats, int max_tries)
{
    geom g;
    int64_t i;
    if (check_dims(L) || mu < 0 || mu > 3 || !(beta > 0.0) || max_tries < 1) return -1;
    if (geom_init(&g, L)) return -2;
    for (i = 0; i < n; i++) {
        if (sites[i] < 0 || sites[i] >= g.V) { geom_free(&g); return -1; }
    }
    for (i = 0; i < n; i++)
        store_link(U, sites[i], mu, update_link(&g, U, beta, seed, t, sites[i], mu, f32, max_tries, stats, NULL), f32);
    geom_free(&g);
    return 0;
}

/* Like oracle_update_links but returns the updated links in `out` (18 doubles
 * each) and leaves U untouched: every update sees the same configuration.
 * margins (may be NULL) receives, per link and subgroup, u3^2 - (1 - delta/2):
 * the one-hit proposal is accepted iff it is <= 0 (NaN for a skipped
 * degenerate subgroup). */
int oracle_updated_links(const int L[4], double beta, uint64_t seed, uint64_t t, int mu, const int64_t* sites, int64_t n,
                         int f32, const double* U, double* out, double* margins, int max_tries)
{
    geom g;
    int64_t i;
    if (check_dims(L) || mu < 0 || mu > 3 || !(beta > 0.0) || max_tries < 1) return -1;
    if (geom_init(&g, L)) return -2;
    for (i = 0; i < n; i++) {
        mat3 m;
        int r, c;
        if (sites[i] < 0 || sites[i] >= g.V) { geom_free(&g); return -1; }
        m = update_link(&g, U, beta, seed, t, sites[i], mu, f32, max_tries, NULL, margins ? margins + 3 * i : NULL);
        if (f32) {
            for (r = 0; r < 2; r++)
                for (c = 0; c < 3; c++) {
                    m.e[r][c].re = (double)(float)m.e[r][c].re;
                    m.e[r][c].im = (double)(float)m.e[r][c].im;
                }
            third_row(&m);
        }
        for (r = 0; r < 3; r++)
            for (c = 0; c < 3; c++) {
                out[i * 18 + (r * 3 + c) * 2] = m.e[r][c].re;
                out[i * 18 + (r * 3 + c) * 2 + 1] = m.e[r][c].im;
            }
    }
    geom_free(&g);
    return 0;
}

/* Random gauge transformation U_mu(x) -> g(x) U_mu(x) g(x+mu)^+ with Haar
 * g(x) drawn from Philox tag 2. */
int oracle_gauge_transform(const int L[4], uint64_t seed, double* U)
{
    geom g;
    int64_t s;
    int mu;
    mat3* gx;
    if (check_dims(L)) return -1;
    if (geom_init(&g, L)) return -2;
    gx = (mat3*)malloc(sizeof(mat3) * (size_t)g.V);
    if (!gx) { geom_free(&g); return -2; }
    for (s = 0; s < g.V; s++) gx[s] = haar_su3(seed, s, 0, 2u);
    for (s = 0; s < g.V; s++)
        for (mu = 0; mu < 4; mu++) {
            mat3 u = load_link(U, s, mu, 0);
            mat3 gd = m_dag(&gx[g.up[s * 4 + mu]]);
            mat3 t1 = m_mul(&gx[s], &u);
            mat3 t2 = m_mul(&t1, &gd);
            store_link(U, s, mu, t2, 0);
        }
    free(gx);
    geom_free(&g);
    return 0;
}

/* n independent KP draws at fixed alpha (Philox tag 3, counter
 * (i, call<<4 | try<<6, 0)), each with up to max_tries proposals;
 * out[4*i..4*i+3] = quaternion if accepted[i], else zeros.  tries (may be
 * NULL) receives the number of proposals drawn.  Returns the number accepted. */
int64_t oracle_kp_draws(double alpha, uint64_t seed, int64_t n, double* out, uint8_t* accepted, int max_tries,
                        int64_t* tries)
{
    int64_t i, nacc = 0, ntry = 0;
    for (i = 0; i < n; i++) {
        uint32_t w[4];
        double u[6], a[4] = {0.0, 0.0, 0.0, 0.0};
        int call, ok = 0, tr;
        for (tr = 0; tr < max_tries && !ok; tr++) {
            for (call = 0; call < 3; call++) {
                draw_words(seed, (uint32_t)i, (uint32_t)((call << 4) | (tr << 6)), (uint64_t)(i >> 32), 3u, w);
                u[2 * call] = oracle_u01_f64(w[0], w[1]);
                u[2 * call + 1] = oracle_u01_f64(w[2], w[3]);
            }
            ok = kp_one_hit(alpha, u, a);
            ntry++;
        }
        out[4 * i] = a[0]; out[4 * i + 1] = a[1]; out[4 * i + 2] = a[2]; out[4 * i + 3] = a[3];
        accepted[i] = (uint8_t)ok;
        nacc += ok;
    }
    if (tries) *tries = ntry;
    return nacc;
}
