/*
 * ge_oracle.c -- plain, serial, FP64 CPU oracle of the group explicit (GE)
 * time step for u_t = u_xx (Parand, Zafarvahedian, Hossayni,
 * arXiv:1310.3422, Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library) shares no code, header or constant with it.
 *
 * Notation.  n interior points with 0-based array indices i = 0..n-1; array
 * index i is the paper's mesh node x_{i+1}, nodes x_0 and x_{n+1} are the
 * Dirichlet walls holding beta_l and beta_r (Sec. 2, problem statement; the
 * paper has one wall value beta, two independent values are a superset).
 * r = tau / h^2 (Sec. 2, after Eq. (aa)).
 *
 * The step (Sec. 2, sub-domain decomposition with sub-domain width k = 1):
 *   parity p = s mod 2 of the global step counter s.
 *   p = 0: points are coupled in groups (0,1), (2,3), ...   (the paper's first
 *          row of each pair of steps: Saul'yev A starts at the left wall of
 *          every odd sub-domain, B at the right wall of every even one);
 *   p = 1: groups (1,2), (3,4), ... and point 0 is a singleton (the second
 *          row: the confluence pairs start at x_{2ik+k-1}, x_{2ik+k}).
 *   A point left without a partner at the right end is a singleton too.
 *   Group (i, i+1), old values a = u[i-1], b = u[i], c = u[i+1], d = u[i+2]:
 *     left member  <- Eq. (cc),  right member <- Eq. (dd),
 *   with the prefactor 1/(1+2r): the determinant of the group's 2x2 system.
 *   (The printed prefactor 1/(3(1+2r)) is a transcription error: the four
 *   numerator coefficients of (cc) sum to 1+2r, so only 1/(1+2r) keeps a
 *   constant state constant.)
 *   Left singleton i = 0: Saul'yev A, Eq. (aa), with u_{-1}^{new} = beta_l.
 *   Right singleton i = n-1: Saul'yev B, Eq. (bb), with u_n^{new} = beta_r.
 *   u[-1] and u[n] at the old level are beta_l and beta_r.
 *
 * Rounding.  Every sum of products is evaluated with fused multiply-adds
 * in the order the formula prints its terms: t = c1*a; t = fma(c2,b,t);
 * t = fma(c3,c,t); t = fma(c4,d,t).  Compile with -ffp-contract=off so the
 * compiler adds no contraction of its own.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Coefficients of Eqs. (cc)/(dd) and (aa)/(bb).
 * out[0..3] = (r+r^2, 1-r^2, r-r^2, r^2) / (1+2r)       -- Eq. (cc) order
 * out[4]    = r/(1+r),  out[5] = (1-r)/(1+r)              -- Eqs. (aa)/(bb) */
void ge_oracle_coefficients(double r, double out[6])
{
    double r2 = r * r;
    double det = 1.0 + 2.0 * r;
    out[0] = (r + r2) / det;
    out[1] = (1.0 - r2) / det;
    out[2] = (r - r2) / det;
    out[3] = r2 / det;
    out[4] = r / (1.0 + r);
    out[5] = (1.0 - r) / (1.0 + r);
}

/* One group (lo, lo+1): Eq. (cc) for the left member, Eq. (dd) for the right. */
static void group_update(const double k[6], double a, double b, double c, double d,
                         double *y, double *z)
{
    double t;
    t = k[0] * a;            /* (r+r^2) a   */
    t = fma(k[1], b, t);     /* (1-r^2) b   */
    t = fma(k[2], c, t);     /* (r-r^2) c   */
    t = fma(k[3], d, t);     /* r^2 d       */
    *y = t;
    t = k[3] * a;            /* r^2 a       */
    t = fma(k[2], b, t);     /* (r-r^2) b   */
    t = fma(k[1], c, t);     /* (1-r^2) c   */
    t = fma(k[0], d, t);     /* (r+r^2) d   */
    *z = t;
}

/* Saul'yev A at the left wall / B at the right wall: the new-level neighbour
 * is the wall value w, the old-level far neighbour is f. */
static double singleton_update(const double k[6], double w, double self, double f)
{
    double t;
    t = k[4] * w;            /* r u_wall^{new}      */
    t = fma(k[5], self, t);  /* (1-r) u_i^{old}     */
    t = fma(k[4], f, t);     /* r u_far^{old}       */
    return t;
}

/* One GE step of the given parity, Dirichlet walls.  Reads u_in[0..n-1],
 * writes u_out[0..n-1]; the two arrays must not overlap.
 * Returns 0, or -1 on invalid arguments. */
int ge_oracle_step(int64_t n, double r, double beta_l, double beta_r, int parity,
                   const double *u_in, double *u_out)
{
    double k[6];
    int64_t lo;
    if (n < 1 || !(r > 0.0) || !isfinite(r) || (parity != 0 && parity != 1) ||
        u_in == NULL || u_out == NULL)
        return -1;
    ge_oracle_coefficients(r, k);

    /* groups of this parity */
    for (lo = parity; lo + 1 < n; lo += 2) {
        double a = (lo == 0) ? beta_l : u_in[lo - 1];
        double b = u_in[lo];
        double c = u_in[lo + 1];
        double d = (lo + 2 == n) ? beta_r : u_in[lo + 2];
        group_update(k, a, b, c, d, &u_out[lo], &u_out[lo + 1]);
    }
    /* left singleton: point 0 at parity 1 */
    if (parity == 1) {
        double far = (n == 1) ? beta_r : u_in[1];
        u_out[0] = singleton_update(k, beta_l, u_in[0], far);
    }
    /* right singleton: the last point when no group covers it */
    if (((n - parity) % 2) == 1) {
        double far = (n == 1) ? beta_l : u_in[n - 2];
        u_out[n - 1] = singleton_update(k, beta_r, u_in[n - 1], far);
    }
    return 0;
}

/* Advance u (in place) by `steps` GE steps starting at global step counter
 * step0 (parity of step s is s mod 2).  Returns 0, or -1 on invalid input or
 * allocation failure. */
int ge_oracle_run(int64_t n, double r, double beta_l, double beta_r, int64_t step0,
                  int64_t steps, double *u)
{
    double *tmp, *src, *dst;
    int64_t s;
    if (n < 1 || steps < 0 || step0 < 0 || u == NULL || !(r > 0.0) || !isfinite(r))
        return -1;
    if (steps == 0)
        return 0;
    tmp = (double *)malloc((size_t)n * sizeof(double));
    if (tmp == NULL)
        return -1;
    src = u;
    dst = tmp;
    for (s = 0; s < steps; ++s) {
        double *t;
        ge_oracle_step(n, r, beta_l, beta_r, (int)((step0 + s) % 2), src, dst);
        t = src;
        src = dst;
        dst = t;
    }
    if (src != u)
        memcpy(u, src, (size_t)n * sizeof(double));
    free(tmp);
    return 0;
}

/* General sub-domain width k (Sec. 2: odd sub-domains [x_{2ik}, x_{2ik+k-1}],
 * even sub-domains [x_{2ik+k}, x_{2(i+1)k-1}] of the paper's nodes x_0..x_{n+1}).
 * Paper node j (array index j-1) lies in sub-domain s = floor(j/k); at parity
 * 0 the odd sub-domains (even s) use Saul'yev A and sweep right from their
 * left wall, the even ones (odd s) use B and sweep left from their right
 * wall; parity 1 swaps the roles.  A B node followed by an A node are the two
 * walls of a confluence: their coupled pair is solved first by Eqs. (cc)/(dd)
 * (the same group formula as k = 1), then the A runs are swept left to right
 * and the B runs right to left, each from its new-level neighbour (the wall
 * value beyond the grid).  k = 1 gives ge_oracle_step bit for bit.
 * Returns 0, or -1 on invalid arguments. */
int ge_oracle_step_k(int64_t n, double r, double beta_l, double beta_r, int parity, int64_t k,
                     const double *u_in, double *u_out)
{
    double kc[6];
    int64_t j;
    char *paired;
    if (n < 1 || k < 1 || !(r > 0.0) || !isfinite(r) || (parity != 0 && parity != 1) ||
        u_in == NULL || u_out == NULL)
        return -1;
    ge_oracle_coefficients(r, kc);
    paired = (char *)calloc((size_t)n + 2, 1);
    if (paired == NULL)
        return -1;
#define OLD(jj) ((jj) == 0 ? beta_l : ((jj) == n + 1 ? beta_r : u_in[(jj) - 1]))
#define ROLE_A(jj) ((((jj) / k) + parity) % 2 == 0)
    /* confluence pairs: B at node j, A at node j+1 (paper nodes 1..n) */
    for (j = 1; j < n; ++j) {
        if (!ROLE_A(j) && ROLE_A(j + 1)) {
            group_update(kc, OLD(j - 1), OLD(j), OLD(j + 1), OLD(j + 2), &u_out[j - 1], &u_out[j]);
            paired[j] = paired[j + 1] = 1;
        }
    }
    /* Saul'yev A runs, left to right from the new left neighbour */
    for (j = 1; j <= n; ++j) {
        if (ROLE_A(j) && !paired[j]) {
            double left_new = (j == 1) ? beta_l : u_out[j - 2];
            u_out[j - 1] = singleton_update(kc, left_new, u_in[j - 1], OLD(j + 1));
        }
    }
    /* Saul'yev B runs, right to left from the new right neighbour */
    for (j = n; j >= 1; --j) {
        if (!ROLE_A(j) && !paired[j]) {
            double right_new = (j == n) ? beta_r : u_out[j];
            u_out[j - 1] = singleton_update(kc, right_new, u_in[j - 1], OLD(j - 1));
        }
    }
#undef OLD
#undef ROLE_A
    free(paired);
    return 0;
}

int ge_oracle_run_k(int64_t n, double r, double beta_l, double beta_r, int64_t k, int64_t step0,
                    int64_t steps, double *u)
{
    double *tmp, *src, *dst;
    int64_t s;
    if (n < 1 || k < 1 || steps < 0 || step0 < 0 || u == NULL || !(r > 0.0) || !isfinite(r))
        return -1;
    if (steps == 0)
        return 0;
    tmp = (double *)malloc((size_t)n * sizeof(double));
    if (tmp == NULL)
        return -1;
    src = u;
    dst = tmp;
    for (s = 0; s < steps; ++s) {
        double *t;
        if (ge_oracle_step_k(n, r, beta_l, beta_r, (int)((step0 + s) % 2), k, src, dst) != 0) {
            free(tmp);
            return -1;
        }
        t = src;
        src = dst;
        dst = t;
    }
    if (src != u)
        memcpy(u, src, (size_t)n * sizeof(double));
    free(tmp);
    return 0;
}

/* Periodic variant (test-only, for the Fourier pin): n even, indices taken
 * modulo n, parity 0 groups (0,1),(2,3),..., parity 1 groups (1,2),...,(n-1,0).
 * No walls, no singletons; the same group formula as the Dirichlet step. */
int ge_oracle_step_periodic(int64_t n, double r, int parity, const double *u_in,
                            double *u_out)
{
    double k[6];
    int64_t lo;
    if (n < 2 || (n % 2) != 0 || !(r > 0.0) || !isfinite(r) ||
        (parity != 0 && parity != 1) || u_in == NULL || u_out == NULL)
        return -1;
    ge_oracle_coefficients(r, k);
    for (lo = parity; lo < n + parity; lo += 2) {
        int64_t im1 = (lo - 1 + n) % n, i0 = lo % n, i1 = (lo + 1) % n, i2 = (lo + 2) % n;
        group_update(k, u_in[im1], u_in[i0], u_in[i1], u_in[i2], &u_out[i0], &u_out[i1]);
    }
    return 0;
}

int ge_oracle_run_periodic(int64_t n, double r, int64_t step0, int64_t steps, double *u)
{
    double *tmp, *src, *dst;
    int64_t s;
    if (n < 2 || (n % 2) != 0 || steps < 0 || step0 < 0 || u == NULL)
        return -1;
    if (steps == 0)
        return 0;
    tmp = (double *)malloc((size_t)n * sizeof(double));
    if (tmp == NULL)
        return -1;
    src = u;
    dst = tmp;
    for (s = 0; s < steps; ++s) {
        double *t;
        if (ge_oracle_step_periodic(n, r, (int)((step0 + s) % 2), src, dst) != 0) {
            free(tmp);
            return -1;
        }
        t = src;
        src = dst;
        dst = t;
    }
    if (src != u)
        memcpy(u, src, (size_t)n * sizeof(double));
    free(tmp);
    return 0;
}
