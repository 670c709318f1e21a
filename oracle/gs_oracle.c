/*
 * Gray-Scott CPU oracle — TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, FP64 restatement of what the GPU path computes, used by the
 * test suite, by the smoke check and by the benchmark's CPU-baseline leg to
 * check the CUDA kernels.  Nothing in the product library may link, load or
 * call this file; it shares no code, header or constant table with the CUDA
 * sources (it re-derives everything from the paper and from the published
 * definitions cited below).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (contraction off so
 * that every a*b+c is two correctly rounded operations, in the order written).
 *
 * Contents
 *   oracle_fmix32          MurmurHash3 32-bit finaliser (Appleby, public domain)
 *   oracle_noise_r         the per-cell, per-step uniform r in (-1,1) of Eq. (1a)
 *   oracle_init            centred-cube initial state
 *   oracle_step            n forward-Euler steps of Eq. (2a,2b) with the
 *                          7-point Laplacian of Eq. (3) and periodic wrap
 *   oracle_window          the same steps for a few sampled cells of a large
 *                          grid, from their light cone only
 *   oracle_conv3d_*        circular 3x3x3 convolution and its two gradients
 *                          (surrogate model; not in the paper)
 *   oracle_bf16_round      bfloat16 round-to-nearest-even of a binary32 value
 *
 * Parity status of each function is stated beside it; every one is pinned by
 * a test in tests/test_oracle_pins.py.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Threads (timing only: every loop below writes disjoint cells, so results  */
/* do not depend on the thread count).                                        */
/* ------------------------------------------------------------------------ */
int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Noise r (Eq. 1a: "r is a uniformly distributed random number between -1  */
/* and 1 for each time and spatial coordinate").  The paper draws it from a  */
/* device RNG; here it is a counter-based hash of (seed, step, cell) so the  */
/* oracle reproduces the GPU's draws exactly.                                 */
/*                                                                            */
/* fmix32 is the MurmurHash3 finaliser as published by A. Appleby           */
/* (smhasher, public domain).  The keyed two-round construction:             */
/*   k1 = fmix32(lo32(seed) ^ fmix32(t ^ 0x9E3779B9))                         */
/*   k2 = fmix32(hi32(seed) ^ fmix32(k1 ^ 0x7F4A7C15))                        */
/*   h  = fmix32(fmix32(c ^ k1) ^ k2),  m = h >> 8  (24 bits)                 */
/*   r  = (2m + 1 - 2^24) / 2^24                                              */
/* r is exact in binary32 and binary64 and lies strictly inside (-1, 1).     */
/* Pinned: MurmurHash3 published vectors; independent numpy restatement;    */
/* the exact distribution of r over all 2^24 codes.                          */
/* ------------------------------------------------------------------------ */
uint32_t oracle_fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

static void step_keys(uint64_t seed, int64_t t, uint32_t* k1, uint32_t* k2)
{
    uint32_t s_lo = (uint32_t)(seed & 0xffffffffu);
    uint32_t s_hi = (uint32_t)(seed >> 32);
    uint32_t a = oracle_fmix32(s_lo ^ oracle_fmix32((uint32_t)t ^ 0x9E3779B9u));
    uint32_t b = oracle_fmix32(s_hi ^ oracle_fmix32(a ^ 0x7F4A7C15u));
    *k1 = a;
    *k2 = b;
}

static double code_to_r(uint32_t h)
{
    int32_t m = (int32_t)(h >> 8);                      /* 0 .. 2^24-1 */
    int32_t num = 2 * m + 1 - (1 << 24);               /* odd, |num| < 2^24 */
    return (double)num / 16777216.0;                    /* exact */
}

double oracle_noise_r(uint64_t seed, int64_t t, uint32_t c)
{
    uint32_t k1, k2;
    step_keys(seed, t, &k1, &k2);
    return code_to_r(oracle_fmix32(oracle_fmix32(c ^ k1) ^ k2));
}

/* r for cells 0..n-1 of step t (used to compare against the GPU's draws). */
void oracle_noise_field(uint64_t seed, int64_t t, int64_t n, double* r)
{
    uint32_t k1, k2;
    step_keys(seed, t, &k1, &k2);
    for (int64_t c = 0; c < n; ++c)
        r[c] = code_to_r(oracle_fmix32(oracle_fmix32((uint32_t)c ^ k1) ^ k2));
}

/* ------------------------------------------------------------------------ */
/* Initial state.  The paper does not print one; the workload defines it:    */
/* u = 1, v = 0 everywhere except a centred cube of side 6,                  */
/* [L/2-3, L/2+3) in each axis (clipped to the grid), where u = 0.25 and     */
/* v = 0.33.  Layout x-fastest: index = x + L*(y + L*z).                     */
/* Pinned: octahedral symmetry and light-cone tests start from it.           */
/* ------------------------------------------------------------------------ */
static int64_t wrap_axis(int64_t i, int L) { return ((i % L) + L) % L; }

static int in_cube(int L, int i)
{
    int lo = L / 2 - 3;
    return i >= lo && i < lo + 6;
}

void oracle_init(int L, double* u, double* v)
{
    for (int z = 0; z < L; ++z)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                int64_t i = (int64_t)x + (int64_t)L * ((int64_t)y + (int64_t)L * z);
                if (in_cube(L, x) && in_cube(L, y) && in_cube(L, z)) {
                    u[i] = 0.25;
                    v[i] = 0.33;
                } else {
                    u[i] = 1.0;
                    v[i] = 0.0;
                }
            }
}

/* ------------------------------------------------------------------------ */
/* Time stepping.                                                             */
/*   Eq. (3):  lap f = -f + (1/6) * (sum of the 6 face neighbours), written  */
/*             as (s - 6 f) / 6 with s summed x-, x+, y-, y+, z-, z+ left to */
/*             right (the operation order of the paper's kernel listing).    */
/*   Eq. (1a): du = Du lap u - u v^2 + F (1 - u) + n r                        */
/*   Eq. (1b): dv = Dv lap v + u v^2 - (F + k) v                              */
/*   Eq. (2):  u' = u + dt du,  v' = v + dt dv   (forward Euler)             */
/* Periodic wrap in every axis (neighbour index (i +- 1 + L) mod L); new     */
/* values go to separate buffers (double buffering, Section 3.2).            */
/* Step t -> t+1 draws r(seed, t, cell).  Fields are updated in place on     */
/* return (u, v hold the state after nsteps).                                 */
/* Pinned: fixed point, symmetry, sine-mode closed form, brute force,        */
/* light cone, translation equivariance, conservation.                       */
/* ------------------------------------------------------------------------ */
static void one_step(int L, const double* u, const double* v, double* un, double* vn,
                     double Du, double Dv, double F, double k, double dt, double noise,
                     uint64_t seed, int64_t t)
{
    uint32_t k1, k2;
    step_keys(seed, t, &k1, &k2);
    const int64_t LL = (int64_t)L * L;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < L; ++z) {
        int zm = (z + L - 1) % L, zp = (z + 1) % L;
        for (int y = 0; y < L; ++y) {
            int ym = (y + L - 1) % L, yp = (y + 1) % L;
            for (int x = 0; x < L; ++x) {
                int xm = (x + L - 1) % L, xp = (x + 1) % L;
                int64_t c   = x  + (int64_t)L * y  + LL * z;
                int64_t cxm = xm + (int64_t)L * y  + LL * z;
                int64_t cxp = xp + (int64_t)L * y  + LL * z;
                int64_t cym = x  + (int64_t)L * ym + LL * z;
                int64_t cyp = x  + (int64_t)L * yp + LL * z;
                int64_t czm = x  + (int64_t)L * y  + LL * zm;
                int64_t czp = x  + (int64_t)L * y  + LL * zp;

                double uc = u[c], vc = v[c];
                double su = u[cxm] + u[cxp];
                su = su + u[cym];
                su = su + u[cyp];
                su = su + u[czm];
                su = su + u[czp];
                double sv = v[cxm] + v[cxp];
                sv = sv + v[cym];
                sv = sv + v[cyp];
                sv = sv + v[czm];
                sv = sv + v[czp];
                double lapu = (su - 6.0 * uc) / 6.0;
                double lapv = (sv - 6.0 * vc) / 6.0;

                double r = code_to_r(oracle_fmix32(oracle_fmix32((uint32_t)c ^ k1) ^ k2));
                double uvv = uc * (vc * vc);
                double du = Du * lapu - uvv;
                du = du + F * (1.0 - uc);
                du = du + noise * r;
                double dv = Dv * lapv + uvv;
                dv = dv - (F + k) * vc;

                un[c] = uc + du * dt;
                vn[c] = vc + dv * dt;
            }
        }
    }
}

/* Returns 0 on success, -1 on a bad argument, -2 when the work buffers cannot
 * be allocated. */
int oracle_step(int L, double* u, double* v, double Du, double Dv, double F, double k,
                double dt, double noise, uint64_t seed, int64_t t0, int64_t nsteps)
{
    if (L < 1 || nsteps < 0) return -1;
    if (nsteps == 0) return 0;
    int64_t n = (int64_t)L * L * L;
    double* un = (double*)malloc((size_t)n * sizeof(double));
    double* vn = (double*)malloc((size_t)n * sizeof(double));
    if (!un || !vn) {
        free(un);
        free(vn);
        return -2;
    }
    double *a = u, *b = v, *c = un, *d = vn;
    for (int64_t s = 0; s < nsteps; ++s) {
        one_step(L, a, b, c, d, Du, Dv, F, k, dt, noise, seed, t0 + s);
        double* tmp;
        tmp = a; a = c; c = tmp;
        tmp = b; b = d; d = tmp;
    }
    if (a != u) {
        memcpy(u, a, (size_t)n * sizeof(double));
        memcpy(v, b, (size_t)n * sizeof(double));
    }
    free(un);
    free(vn);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The paper's own kernel variants (Listing 2; bandwidth study, Section 5.1, */
/* Tables 2-3).                                                               */
/*                                                                            */
/* Held outer layer: the paper's kernel returns without writing for a cell   */
/* whose index lies on the first or last layer of any axis (on the full     */
/* domain those faces are ghost cells filled by the MPI exchange).  On one   */
/* grid with no neighbours the reading taken is: those cells keep their     */
/* values, and every other cell updates by Eq. 1-3 exactly as in            */
/* oracle_step (its six neighbours are all inside the grid, so nothing      */
/* wraps).  The noise draw of an interior cell is the same r(seed, t, c).    */
/*                                                                            */
/* "1-variable, no random" (Table 2): one field, no reaction and no noise,   */
/*   f' = f + dt (D lap f),  lap f = (s - 6 f) / 6  (Eq. 3, same order),     */
/* with either periodic wrap or the held outer layer.                        */
/*                                                                            */
/* Pinned: boundary cells unchanged; Dirichlet sine modes                    */
/* sin(pi m i / (L-1)) vanish on both held faces and decay by the closed-    */
/* form factor; periodic sine modes; conservation; brute force on tiny       */
/* grids.                                                                     */
/* ------------------------------------------------------------------------ */
static int on_face(int L, int x, int y, int z)
{
    return x == 0 || y == 0 || z == 0 || x == L - 1 || y == L - 1 || z == L - 1;
}

static void one_step_held(int L, const double* u, const double* v, double* un, double* vn, double Du, double Dv,
                          double F, double k, double dt, double noise, uint64_t seed, int64_t t)
{
    uint32_t k1, k2;
    step_keys(seed, t, &k1, &k2);
    const int64_t LL = (int64_t)L * L;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < L; ++z) {
        for (int y = 0; y < L; ++y) {
            for (int x = 0; x < L; ++x) {
                const int64_t c = x + (int64_t)L * y + LL * z;
                if (on_face(L, x, y, z)) {
                    un[c] = u[c];
                    vn[c] = v[c];
                    continue;
                }
                const double uc = u[c], vc = v[c];
                double su = u[c - 1] + u[c + 1];
                su = su + u[c - L];
                su = su + u[c + L];
                su = su + u[c - LL];
                su = su + u[c + LL];
                double sv = v[c - 1] + v[c + 1];
                sv = sv + v[c - L];
                sv = sv + v[c + L];
                sv = sv + v[c - LL];
                sv = sv + v[c + LL];
                const double lapu = (su - 6.0 * uc) / 6.0;
                const double lapv = (sv - 6.0 * vc) / 6.0;
                const double r = code_to_r(oracle_fmix32(oracle_fmix32((uint32_t)c ^ k1) ^ k2));
                const double uvv = uc * (vc * vc);
                double du = Du * lapu - uvv;
                du = du + F * (1.0 - uc);
                du = du + noise * r;
                double dv = Dv * lapv + uvv;
                dv = dv - (F + k) * vc;
                un[c] = uc + du * dt;
                vn[c] = vc + dv * dt;
            }
        }
    }
}

/* Two fields, held outer layer.  Returns 0, -1 (bad argument), -2 (memory). */
int oracle_step_held(int L, double* u, double* v, double Du, double Dv, double F, double k, double dt,
                     double noise, uint64_t seed, int64_t t0, int64_t nsteps)
{
    if (L < 1 || nsteps < 0) return -1;
    if (nsteps == 0) return 0;
    const int64_t n = (int64_t)L * L * L;
    double* un = (double*)malloc((size_t)n * sizeof(double));
    double* vn = (double*)malloc((size_t)n * sizeof(double));
    if (!un || !vn) {
        free(un);
        free(vn);
        return -2;
    }
    double *a = u, *b = v, *c = un, *d = vn;
    for (int64_t s = 0; s < nsteps; ++s) {
        one_step_held(L, a, b, c, d, Du, Dv, F, k, dt, noise, seed, t0 + s);
        double* tmp;
        tmp = a; a = c; c = tmp;
        tmp = b; b = d; d = tmp;
    }
    if (a != u) {
        memcpy(u, a, (size_t)n * sizeof(double));
        memcpy(v, b, (size_t)n * sizeof(double));
    }
    free(un);
    free(vn);
    return 0;
}

/* One field, f' = f + dt (D lap f); held = 0: periodic wrap, 1: held outer
 * layer.  Returns 0, -1 (bad argument), -2 (memory). */
int oracle_diffuse(int L, double* f, double D, double dt, int held, int64_t nsteps)
{
    if (L < 1 || nsteps < 0 || (held != 0 && held != 1)) return -1;
    if (nsteps == 0) return 0;
    const int64_t n = (int64_t)L * L * L, LL = (int64_t)L * L;
    double* g = (double*)malloc((size_t)n * sizeof(double));
    if (!g) return -2;
    double *a = f, *b = g;
    for (int64_t s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
        for (int z = 0; z < L; ++z) {
            const int zm = (z + L - 1) % L, zp = (z + 1) % L;
            for (int y = 0; y < L; ++y) {
                const int ym = (y + L - 1) % L, yp = (y + 1) % L;
                for (int x = 0; x < L; ++x) {
                    const int xm = (x + L - 1) % L, xp = (x + 1) % L;
                    const int64_t c = x + (int64_t)L * y + LL * z;
                    if (held && on_face(L, x, y, z)) {
                        b[c] = a[c];
                        continue;
                    }
                    double sum = a[xm + (int64_t)L * y + LL * z] + a[xp + (int64_t)L * y + LL * z];
                    sum = sum + a[x + (int64_t)L * ym + LL * z];
                    sum = sum + a[x + (int64_t)L * yp + LL * z];
                    sum = sum + a[x + (int64_t)L * y + LL * zm];
                    sum = sum + a[x + (int64_t)L * y + LL * zp];
                    const double lap = (sum - 6.0 * a[c]) / 6.0;
                    b[c] = a[c] + dt * (D * lap);
                }
            }
        }
        double* tmp = a;
        a = b;
        b = tmp;
    }
    if (a != f) memcpy(f, a, (size_t)n * sizeof(double));
    free(g);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sampled cells of a large run.  The state of a cell after n steps depends  */
/* only on cells within n steps of it (one neighbour per step), so the       */
/* cells of a (2m+1)^3 cube centred at (cx, cy, cz) can be computed from a   */
/* window of radius R = n + m of the periodic L^3 grid.  Window cell (i,j,l) */
/* is global cell ((cx-R+i) mod L, (cy-R+j) mod L, (cz-R+l) mod L); the noise */
/* uses the global cell index.  Step s updates only window cells at least    */
/* s+1 from the window border (the rest would need cells outside it), with   */
/* the same arithmetic as one_step.  Start state: the centred cube           */
/* (u0 == NULL) or the full arrays u0, v0 of the grid.                        */
/* Output: uo, vo of (2m+1)^3 cells, x-fastest.  Returns 0, or -1/-2.        */
/* Pinned: equals oracle_step at the sampled cells (tests).                  */
/* ------------------------------------------------------------------------ */
int oracle_window(int L, int cx, int cy, int cz, int m, const double* u0, const double* v0,
                  double Du, double Dv, double F, double k, double dt, double noise,
                  uint64_t seed, int64_t t0, int nsteps, double* uo, double* vo)
{
    if (L < 1 || m < 0 || nsteps < 0) return -1;
    const int R = nsteps + m;
    const int W = 2 * R + 1;
    const int64_t WW = (int64_t)W * W, n = WW * W;
    double* a = (double*)malloc((size_t)n * sizeof(double));
    double* b = (double*)malloc((size_t)n * sizeof(double));
    double* c2 = (double*)malloc((size_t)n * sizeof(double));
    double* d = (double*)malloc((size_t)n * sizeof(double));
    uint32_t* gid = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    if (!a || !b || !c2 || !d || !gid) {
        free(a); free(b); free(c2); free(d); free(gid);
        return -2;
    }
    for (int l = 0; l < W; ++l)
        for (int j = 0; j < W; ++j)
            for (int i = 0; i < W; ++i) {
                int gx = (int)wrap_axis(cx - R + i, L);
                int gy = (int)wrap_axis(cy - R + j, L);
                int gz = (int)wrap_axis(cz - R + l, L);
                int64_t g = gx + (int64_t)L * (gy + (int64_t)L * gz);
                int64_t w = i + (int64_t)W * j + WW * l;
                gid[w] = (uint32_t)g;
                if (u0) {
                    a[w] = u0[g];
                    b[w] = v0[g];
                } else if (in_cube(L, gx) && in_cube(L, gy) && in_cube(L, gz)) {
                    a[w] = 0.25;
                    b[w] = 0.33;
                } else {
                    a[w] = 1.0;
                    b[w] = 0.0;
                }
            }
    memcpy(c2, a, (size_t)n * sizeof(double));
    memcpy(d, b, (size_t)n * sizeof(double));
    for (int s = 0; s < nsteps; ++s) {
        uint32_t k1, k2;
        step_keys(seed, t0 + s, &k1, &k2);
        const int lo = s + 1, hi = W - 2 - s;
        for (int l = lo; l <= hi; ++l)
            for (int j = lo; j <= hi; ++j)
                for (int i = lo; i <= hi; ++i) {
                    int64_t w = i + (int64_t)W * j + WW * l;
                    double uc = a[w], vc = b[w];
                    double su = a[w - 1] + a[w + 1];
                    su = su + a[w - W];
                    su = su + a[w + W];
                    su = su + a[w - WW];
                    su = su + a[w + WW];
                    double sv = b[w - 1] + b[w + 1];
                    sv = sv + b[w - W];
                    sv = sv + b[w + W];
                    sv = sv + b[w - WW];
                    sv = sv + b[w + WW];
                    double lapu = (su - 6.0 * uc) / 6.0;
                    double lapv = (sv - 6.0 * vc) / 6.0;
                    double r = code_to_r(oracle_fmix32(oracle_fmix32(gid[w] ^ k1) ^ k2));
                    double uvv = uc * (vc * vc);
                    double du = Du * lapu - uvv;
                    du = du + F * (1.0 - uc);
                    du = du + noise * r;
                    double dv = Dv * lapv + uvv;
                    dv = dv - (F + k) * vc;
                    c2[w] = uc + du * dt;
                    d[w] = vc + dv * dt;
                }
        /* copy the updated interior back (border cells keep stale values and
           are never read by a later step's smaller interior) */
        for (int l = lo; l <= hi; ++l)
            for (int j = lo; j <= hi; ++j)
                for (int i = lo; i <= hi; ++i) {
                    int64_t w = i + (int64_t)W * j + WW * l;
                    a[w] = c2[w];
                    b[w] = d[w];
                }
    }
    const int side = 2 * m + 1;
    for (int l = 0; l < side; ++l)
        for (int j = 0; j < side; ++j)
            for (int i = 0; i < side; ++i) {
                int64_t w = (nsteps + i) + (int64_t)W * (nsteps + j) + WW * (nsteps + l);
                int64_t o = i + (int64_t)side * (j + (int64_t)side * l);
                uo[o] = a[w];
                vo[o] = b[w];
            }
    free(a); free(b); free(c2); free(d); free(gid);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Surrogate model primitives (not in the paper).                             */
/*                                                                            */
/* Circular 3x3x3 convolution, channels-last.  For a batch of N periodic     */
/* L^3 grids:                                                                 */
/*   y[n,z,y,x,co] = b[co] + sum_{tap, ci} w[tap, ci, co] *                   */
/*                   x[n, (z+dz) mod L, (y+dy) mod L, (x+dx) mod L, ci]       */
/* with tap = 9 (dz+1) + 3 (dy+1) + (dx+1), dz, dy, dx in {-1, 0, 1}.        */
/* bwd_data:   dx[n,p,ci] = sum_{tap,co} w[tap,ci,co] * dy[n, p - d(tap), co] */
/* bwd_weight: dw[tap,ci,co] = sum_{n,p} x[n, p + d(tap), ci] * dy[n,p,co]   */
/*             db[co] = sum_{n,p} dy[n,p,co]                                  */
/* (the two gradients are the transposes of the forward map, written out).  */
/* Pinned: FFT circular convolution, single-tap shifts, adjoint identity     */
/* <conv(x), g> = <x, bwd_data(g)>, finite differences.                      */
/* ------------------------------------------------------------------------ */
static int64_t wrapi(int64_t i, int L) { return ((i % L) + L) % L; }

static int64_t cell_at(int L, int64_t z, int64_t y, int64_t x)
{
    return wrapi(x, L) + (int64_t)L * (wrapi(y, L) + (int64_t)L * wrapi(z, L));
}

void oracle_conv3d_fwd(int N, int L, int Cin, int Cout, const double* x, const double* w,
                       const double* b, double* y)
{
    const int64_t cells = (int64_t)L * L * L;
#pragma omp parallel for collapse(2) schedule(static)
    for (int n = 0; n < N; ++n)
        for (int z = 0; z < L; ++z)
            for (int yy = 0; yy < L; ++yy)
                for (int xx = 0; xx < L; ++xx) {
                    int64_t p = xx + (int64_t)L * (yy + (int64_t)L * z);
                    double* out = y + ((int64_t)n * cells + p) * Cout;
                    for (int co = 0; co < Cout; ++co) out[co] = b ? b[co] : 0.0;
                    for (int dz = -1; dz <= 1; ++dz)
                        for (int dy = -1; dy <= 1; ++dy)
                            for (int dx = -1; dx <= 1; ++dx) {
                                int tap = 9 * (dz + 1) + 3 * (dy + 1) + (dx + 1);
                                int64_t q = cell_at(L, z + dz, yy + dy, xx + dx);
                                const double* in = x + ((int64_t)n * cells + q) * Cin;
                                for (int ci = 0; ci < Cin; ++ci)
                                    for (int co = 0; co < Cout; ++co)
                                        out[co] += w[((int64_t)tap * Cin + ci) * Cout + co] * in[ci];
                            }
                }
}

void oracle_conv3d_bwd_data(int N, int L, int Cin, int Cout, const double* dy, const double* w,
                            double* dx)
{
    const int64_t cells = (int64_t)L * L * L;
#pragma omp parallel for collapse(2) schedule(static)
    for (int n = 0; n < N; ++n)
        for (int z = 0; z < L; ++z)
            for (int yy = 0; yy < L; ++yy)
                for (int xx = 0; xx < L; ++xx) {
                    int64_t p = xx + (int64_t)L * (yy + (int64_t)L * z);
                    double* out = dx + ((int64_t)n * cells + p) * Cin;
                    for (int ci = 0; ci < Cin; ++ci) out[ci] = 0.0;
                    /* input cell p feeds output cell p - d with tap d */
                    for (int dz = -1; dz <= 1; ++dz)
                        for (int dyo = -1; dyo <= 1; ++dyo)
                            for (int dxo = -1; dxo <= 1; ++dxo) {
                                int tap = 9 * (dz + 1) + 3 * (dyo + 1) + (dxo + 1);
                                int64_t q = cell_at(L, z - dz, yy - dyo, xx - dxo);
                                const double* g = dy + ((int64_t)n * cells + q) * Cout;
                                for (int ci = 0; ci < Cin; ++ci)
                                    for (int co = 0; co < Cout; ++co)
                                        out[ci] += w[((int64_t)tap * Cin + ci) * Cout + co] * g[co];
                            }
                }
}

void oracle_conv3d_bwd_weight(int N, int L, int Cin, int Cout, const double* x, const double* dy,
                              double* dw, double* db)
{
    const int64_t cells = (int64_t)L * L * L;
    memset(dw, 0, sizeof(double) * 27 * (size_t)Cin * Cout);
    if (db) memset(db, 0, sizeof(double) * (size_t)Cout);
    for (int n = 0; n < N; ++n)
        for (int z = 0; z < L; ++z)
            for (int yy = 0; yy < L; ++yy)
                for (int xx = 0; xx < L; ++xx) {
                    int64_t p = xx + (int64_t)L * (yy + (int64_t)L * z);
                    const double* g = dy + ((int64_t)n * cells + p) * Cout;
                    if (db)
                        for (int co = 0; co < Cout; ++co) db[co] += g[co];
                    for (int dz = -1; dz <= 1; ++dz)
                        for (int dyo = -1; dyo <= 1; ++dyo)
                            for (int dxo = -1; dxo <= 1; ++dxo) {
                                int tap = 9 * (dz + 1) + 3 * (dyo + 1) + (dxo + 1);
                                int64_t q = cell_at(L, z + dz, yy + dyo, xx + dxo);
                                const double* in = x + ((int64_t)n * cells + q) * Cin;
                                for (int ci = 0; ci < Cin; ++ci)
                                    for (int co = 0; co < Cout; ++co)
                                        dw[((int64_t)tap * Cin + ci) * Cout + co] += in[ci] * g[co];
                            }
                }
}

/* ------------------------------------------------------------------------ */
/* bfloat16 rounding (IEEE binary32 with the low 16 mantissa bits dropped,   */
/* round to nearest, ties to even; NaN kept quiet).  Returns the rounded     */
/* value widened back to double.  Input is first rounded to binary32, as the */
/* GPU path stores FP32 values before casting.                                */
/* Pinned: against PyTorch's bfloat16 conversion and hand-checked ties.      */
/* ------------------------------------------------------------------------ */
void oracle_bf16_round(int64_t n, const double* in, double* out)
{
    for (int64_t i = 0; i < n; ++i) {
        float f = (float)in[i];
        uint32_t bits;
        memcpy(&bits, &f, 4);
        if ((bits & 0x7f800000u) == 0x7f800000u && (bits & 0x007fffffu)) {
            bits |= 0x00400000u; /* quiet NaN */
            bits &= 0xffff0000u;
        } else {
            uint32_t lsb = (bits >> 16) & 1u;
            bits += 0x7fffu + lsb;
            bits &= 0xffff0000u;
        }
        memcpy(&f, &bits, 4);
        out[i] = (double)f;
    }
}
