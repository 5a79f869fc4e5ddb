/*
 * Oracle (test infrastructure only): the Wilson-Dirac operator in plain C,
 * double-precision complex, written as the definition reads.  Nothing of the
 * CUDA library is used here, and the library uses nothing of this file.
 *
 * Paper, Section 3: the test problem is Wilson fermions at hopping parameter
 * kappa; the operator's formula is not printed, so the standard form is
 * taken (Wilson r = 1):
 *
 *   (D psi)(x) = psi(x) - kappa * sum_{mu=0..3} [ (1 - g_mu) U_mu(x) psi(x+mu) s+
 *                                             + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu) s- ]
 *
 * s+/s- = -1 on a hop that wraps the t direction (antiperiodic in time),
 * +1 otherwise (periodic in space).  D^dag = g5 D g5 with g5 = g1 g2 g3 g4,
 * which the tests check against the adjoint definition <phi, D psi> = <D^dag phi, psi>.
 *
 * Layouts: site s = x + Lx*(y + Ly*(z + Lz*t)); spinor [site][spin][colour];
 * gauge [site][mu][a][b]; all double complex (re, im interleaved).
 * The gamma matrices are the chiral (Weyl) Euclidean basis
 *   g_k = [[0, -i sigma_k], [i sigma_k, 0]] (k = 1,2,3),  g_4 = [[0, 1], [1, 0]].
 */
#include <complex.h>
#include <stddef.h>
#include <string.h>

typedef double complex cplx;

static const cplx GAMMA[4][4][4] = {
    /* g1 (x) */
    {{0, 0, 0, -I}, {0, 0, -I, 0}, {0, I, 0, 0}, {I, 0, 0, 0}},
    /* g2 (y) */
    {{0, 0, 0, -1}, {0, 0, 1, 0}, {0, 1, 0, 0}, {-1, 0, 0, 0}},
    /* g3 (z) */
    {{0, 0, -I, 0}, {0, 0, 0, I}, {I, 0, 0, 0}, {0, -I, 0, 0}},
    /* g4 (t) */
    {{0, 0, 1, 0}, {0, 0, 0, 1}, {1, 0, 0, 0}, {0, 1, 0, 0}},
};

/* Copy out the gamma table (mu = 0..3) the operator uses, for the tests. */
void oracle_gamma(int mu, double *out /* 16 complex = 32 doubles */)
{
    memcpy(out, GAMMA[mu], sizeof(cplx) * 16);
}

/* g5 = g1 g2 g3 g4, formed by matrix products (not typed in). */
static void gamma5(cplx g5[4][4])
{
    cplx a[4][4], b[4][4];
    memcpy(a, GAMMA[0], sizeof(a));
    for (int m = 1; m < 4; m++) {
        for (int i = 0; i < 4; i++)
            for (int j = 0; j < 4; j++) {
                cplx s = 0;
                for (int k = 0; k < 4; k++) s += a[i][k] * GAMMA[m][k][j];
                b[i][j] = s;
            }
        memcpy(a, b, sizeof(a));
    }
    memcpy(g5, a, sizeof(a));
}

void oracle_gamma5(double *out)
{
    cplx g5[4][4];
    gamma5(g5);
    memcpy(out, g5, sizeof(g5));
}

static void site_coords(const int d[4], long s, int c[4])
{
    c[0] = (int)(s % d[0]); s /= d[0];
    c[1] = (int)(s % d[1]); s /= d[1];
    c[2] = (int)(s % d[2]); s /= d[2];
    c[3] = (int)s;
}

static long site_index(const int d[4], const int c[4])
{
    return c[0] + (long)d[0] * (c[1] + (long)d[1] * (c[2] + (long)d[2] * c[3]));
}

/* out = D in.  `in` and `out` must not alias. */
static void wilson_D(const int d[4], const cplx *U, double kappa, const cplx *in, cplx *out)
{
    long vol = (long)d[0] * d[1] * d[2] * d[3];
#pragma omp parallel for schedule(static) if (vol >= 4096)
    for (long s = 0; s < vol; s++) {
        int c[4];
        site_coords(d, s, c);
        cplx acc[4][3];
        for (int i = 0; i < 4; i++)
            for (int a = 0; a < 3; a++) acc[i][a] = in[(s * 4 + i) * 3 + a];

        for (int mu = 0; mu < 4; mu++) {
            /* forward hop: (1 - g_mu) U_mu(x) psi(x + mu) */
            int cf[4] = {c[0], c[1], c[2], c[3]};
            cf[mu] = (c[mu] + 1) % d[mu];
            double sf = (mu == 3 && c[3] == d[3] - 1) ? -1.0 : 1.0;
            long yf = site_index(d, cf);
            const cplx *Uf = U + ((s * 4 + mu) * 9);
            cplx chi[4][3];
            for (int i = 0; i < 4; i++)
                for (int a = 0; a < 3; a++) {
                    cplx t = 0;
                    for (int b = 0; b < 3; b++) t += Uf[a * 3 + b] * in[(yf * 4 + i) * 3 + b];
                    chi[i][a] = t;
                }
            for (int i = 0; i < 4; i++)
                for (int a = 0; a < 3; a++) {
                    cplx t = 0;
                    for (int j = 0; j < 4; j++) {
                        cplx p = (i == j ? 1.0 : 0.0) - GAMMA[mu][i][j];
                        t += p * chi[j][a];
                    }
                    acc[i][a] -= kappa * sf * t;
                }

            /* backward hop: (1 + g_mu) U_mu(x - mu)^dag psi(x - mu) */
            int cb[4] = {c[0], c[1], c[2], c[3]};
            cb[mu] = (c[mu] + d[mu] - 1) % d[mu];
            double sb = (mu == 3 && c[3] == 0) ? -1.0 : 1.0;
            long yb = site_index(d, cb);
            const cplx *Ub = U + ((yb * 4 + mu) * 9);
            for (int i = 0; i < 4; i++)
                for (int a = 0; a < 3; a++) {
                    cplx t = 0;
                    for (int b = 0; b < 3; b++) t += conj(Ub[b * 3 + a]) * in[(yb * 4 + i) * 3 + b];
                    chi[i][a] = t;
                }
            for (int i = 0; i < 4; i++)
                for (int a = 0; a < 3; a++) {
                    cplx t = 0;
                    for (int j = 0; j < 4; j++) {
                        cplx p = (i == j ? 1.0 : 0.0) + GAMMA[mu][i][j];
                        t += p * chi[j][a];
                    }
                    acc[i][a] -= kappa * sb * t;
                }
        }
        for (int i = 0; i < 4; i++)
            for (int a = 0; a < 3; a++) out[(s * 4 + i) * 3 + a] = acc[i][a];
    }
}

static void apply_g5(long vol, const cplx g5[4][4], const cplx *in, cplx *out)
{
#pragma omp parallel for schedule(static) if (vol >= 4096)
    for (long s = 0; s < vol; s++)
        for (int a = 0; a < 3; a++) {
            cplx t[4];
            for (int i = 0; i < 4; i++) {
                cplx u = 0;
                for (int j = 0; j < 4; j++) u += g5[i][j] * in[(s * 4 + j) * 3 + a];
                t[i] = u;
            }
            for (int i = 0; i < 4; i++) out[(s * 4 + i) * 3 + a] = t[i];
        }
}

/*
 * op = 0: out = D in;  op = 1: out = D^dag in = g5 D g5 in;  op = 2: out = D^dag D in.
 * `tmp` is caller scratch of one spinor field.  in/out/tmp must be distinct.
 */
void oracle_wilson_apply(const int dims[4], const double *U, double kappa, int op,
                         const double *in, double *out, double *tmp)
{
    const cplx *u = (const cplx *)U;
    const cplx *x = (const cplx *)in;
    cplx *y = (cplx *)out;
    cplx *t = (cplx *)tmp;
    long vol = (long)dims[0] * dims[1] * dims[2] * dims[3];
    cplx g5[4][4];
    gamma5(g5);
    if (op == 0) {
        wilson_D(dims, u, kappa, x, y);
    } else if (op == 1) {
        apply_g5(vol, g5, x, t);
        wilson_D(dims, u, kappa, t, y);
        apply_g5(vol, g5, y, y);
    } else {
        wilson_D(dims, u, kappa, x, t);
        apply_g5(vol, g5, t, t);
        wilson_D(dims, u, kappa, t, y);
        apply_g5(vol, g5, y, y);
    }
}
