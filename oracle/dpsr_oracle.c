/*
 * FP64 CPU oracle of the spectral Differentiable Poisson Surface Reconstruction
 * (DPSR) layer of "Shape As Points" (Peng et al., arXiv 2106.03452), forward
 * and backward.
 *
 * THIS IS TEST INFRASTRUCTURE. It exists so that the CUDA path can be checked
 * against a slow, plainly written implementation of what the paper defines.
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it. The GPU library shares no code, header or table with
 * it, and it never calls the GPU library.
 *
 * Every step follows the paper's order and notation:
 *   - point rasterization: inverse trilinear splat of the normals onto the
 *     r^3 grid vertices (Sec. 3.1 "Point Rasterization", Eq. A1-A2);
 *   - forward FFT of the rasterized field (Eq. A3), spectral divergence,
 *     inverse Laplacian and Gaussian smoothing (Eq. 3 / Eq. A7);
 *   - inverse FFT to the unnormalised indicator chi' (Eq. A8);
 *   - shift by the mean of chi' at the points and scale so that
 *     |chi(x=0)| = m = 0.5 (Eq. 2, Eq. 4 / Eq. A9);
 *   - the backward pass is the exact adjoint (reverse-mode derivative) of the
 *     above, which is what the paper obtains from autograd (Eq. 5).
 *
 * Readings where the paper is silent or ambiguous (each is listed in the
 * design notes of the repository):
 *   R1 grid: periodic unit cube [0,1)^3, origin c0 = 0, voxel size s = 1/r,
 *      vertex j sits at j/r; coordinates are wrapped periodically.
 *   R3 frequencies u are integer cycles per unit length: u_a = k_a for
 *      k_a < r/2, k_a - r for k_a > r/2.
 *   R4 the spectral numerator is the dot product u . v~ (Eq. 3), not the
 *      element-wise product printed in Eq. A7.
 *   R5 the DC term of chi~ is zero.
 *   R6 at a Nyquist index k_a = r/2 the a-th term of u . v~ is zero; |u|^2
 *      there uses |u_a| = r/2. This equals taking Re() of a full complex
 *      inverse transform with either sign of u_a.
 *   R7 the scale uses s = chi'(0) - mean, the shifted value at the grid
 *      vertex x = 0, so that |chi(0)| = m holds exactly (Eq. 2).
 *   R8 the scale m/|s| is positive: no sign flip.
 *   R9 the mean is the plain average over all N input points.
 *   R11 when c*r is an integer the floor cell is used; the weight derivative
 *      is the one-sided (right) derivative of that cell.
 *   R12 the backward pass differentiates through the mean and the scale.
 *   R13 a box of side lengths L (voxel size L_d / r, Eq. A1's anisotropic
 *      s): coordinates enter as c_d / L_d, u_d = f_d / L_d, the Gaussian's
 *      sigma stays in grid units along every axis, dL/dc_d = dL/dx_d / L_d.
 *
 * Conventions: points and normals are N x 3 row-major; grids are r^3 in C
 * order g[ix][iy][iz] (iz fastest), axis 0 is the x coordinate. The forward
 * DFT is unnormalised with exponent -2 pi i k.j / r (Eq. A3); the inverse
 * carries 1/r^3 and exponent +2 pi i (Eq. A4).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)
#define ORACLE_EDEGENERATE (-4)

static const double kPi = 3.14159265358979323846264338327950288;
static const double kM = 0.5; /* m of Eq. 2 */

static int is_pow2(int r) { return r >= 2 && (r & (r - 1)) == 0; }

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads for the oracle's parallel loops from now on (n >= 1); for timing
 * the oracle on one core and on all of them. */
void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* 1D complex FFT: textbook iterative radix-2 Cooley-Tukey, in place.        */
/* sign = -1 is the forward transform of Eq. A3, +1 the inverse kernel of    */
/* Eq. A4 (without the 1/n, which the 3D routine applies).                   */
/* tw[k] = exp(sign * 2 pi i k / n) for k < n/2, precomputed by the caller.  */
/* ------------------------------------------------------------------------ */
static void fft1d(cplx *a, int n, const cplx *tw)
{
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            cplx t = a[i];
            a[i] = a[j];
            a[j] = t;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len / 2, step = n / len;
        for (int i = 0; i < n; i += len)
            for (int k = 0; k < half; k++) {
                cplx w = tw[k * step];
                cplx u = a[i + k], v = a[i + k + half] * w;
                a[i + k] = u + v;
                a[i + k + half] = u - v;
            }
    }
}

static void make_twiddles(cplx *tw, int n, int sign)
{
    for (int k = 0; k < n / 2; k++) {
        double ang = sign * 2.0 * kPi * (double)k / (double)n;
        tw[k] = cos(ang) + I * sin(ang);
    }
}

/* 3D DFT over an r^3 complex grid, one axis after the other. inverse = 0:
 * unnormalised forward transform (Eq. A3). inverse = 1: the inverse transform
 * (Eq. A4) including the 1/r^3 factor. */
static int fft3(cplx *g, int r, int inverse)
{
    cplx *tw = malloc(sizeof(cplx) * (size_t)(r / 2 > 0 ? r / 2 : 1));
    if (!tw) return ORACLE_ENOMEM;
    make_twiddles(tw, r, inverse ? +1 : -1);
    const int64_t r2 = (int64_t)r * r;
    int err = 0;
    for (int axis = 0; axis < 3; axis++) {
        /* element stride along the transformed axis */
        const int64_t stride = axis == 0 ? r2 : (axis == 1 ? r : 1);
#pragma omp parallel
        {
            cplx *line = malloc(sizeof(cplx) * (size_t)r);
            if (!line) {
#pragma omp atomic write
                err = 1;
            } else {
#pragma omp for schedule(static)
                for (int64_t p = 0; p < r2; p++) {
                    /* p enumerates the r^2 lines; base = first element */
                    int64_t a = p / r, b = p % r, base;
                    if (axis == 0) base = a * r + b;           /* (., a, b) */
                    else if (axis == 1) base = a * r2 + b;     /* (a, ., b) */
                    else base = a * r2 + b * r;                /* (a, b, .) */
                    for (int i = 0; i < r; i++) line[i] = g[base + i * stride];
                    fft1d(line, r, tw);
                    for (int i = 0; i < r; i++) g[base + i * stride] = line[i];
                }
                free(line);
            }
        }
    }
    free(tw);
    if (err) return ORACLE_ENOMEM;
    if (inverse) {
        const double inv = 1.0 / ((double)r * r2);
        const int64_t n = r2 * r;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++) g[i] *= inv;
    }
    return ORACLE_OK;
}

/* Exported for the FFT pins: g is r^3 interleaved (re, im) doubles. */
int oracle_fft3(int r, double *g, int inverse)
{
    if (!is_pow2(r) || !g) return ORACLE_EINVAL;
    return fft3((cplx *)g, r, inverse);
}

/* ------------------------------------------------------------------------ */
/* Trilinear neighbourhood of one point (Eq. A1, reading R1/R11).           */
/* For axis d: x~ = c_d * r, i0 = floor(x~), t = x~ - i0; the two vertices   */
/* are i0 and i0 + 1 (mod r) with weights 1 - t and t. The weight of vertex  */
/* (i0 + delta) is the product over the three axes; it equals               */
/* T(c, s*j + c0, s) = prod_d max(0, 1 - |c_d - j_d s_d| / s_d).            */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t idx[8];   /* flat grid index of vertex delta = (dx,dy,dz), bit 2,1,0 */
    double w[8];      /* trilinear weight */
    double dw[8][3];  /* d w / d c_d, right derivative on the floor cell */
} stencil;

static int make_stencil(const double *c, int r, stencil *st)
{
    int64_t lo[3], hi[3];
    double t[3];
    for (int d = 0; d < 3; d++) {
        if (!isfinite(c[d])) return ORACLE_EDEGENERATE;
        double x = c[d] * (double)r;
        double f = floor(x);
        if (fabs(f) > 1e15) return ORACLE_EDEGENERATE;
        t[d] = x - f;
        int64_t i0 = (int64_t)f % r;
        if (i0 < 0) i0 += r;
        lo[d] = i0;
        hi[d] = (i0 + 1) % r;
    }
    for (int v = 0; v < 8; v++) {
        int del[3] = {(v >> 2) & 1, (v >> 1) & 1, v & 1};
        int64_t j[3];
        double f[3], df[3];
        for (int d = 0; d < 3; d++) {
            j[d] = del[d] ? hi[d] : lo[d];
            f[d] = del[d] ? t[d] : 1.0 - t[d];
            df[d] = del[d] ? (double)r : -(double)r;
        }
        st->idx[v] = (j[0] * r + j[1]) * r + j[2];
        st->w[v] = f[0] * f[1] * f[2];
        st->dw[v][0] = df[0] * f[1] * f[2];
        st->dw[v][1] = f[0] * df[1] * f[2];
        st->dw[v][2] = f[0] * f[1] * df[2];
    }
    return ORACLE_OK;
}

/* Splat (Eq. A2): grid[ch][j] += sum_i w_ij * vals[i][ch]; grid zeroed here.
 * vals == NULL splats the constant 1 (the weight field W_j = sum_i w_ij). */
static int splat(int r, int64_t N, const double *pts, const double *vals, int nch,
                 double *grid)
{
    const int64_t n = (int64_t)r * r * r;
    memset(grid, 0, sizeof(double) * (size_t)(n * nch));
    for (int64_t i = 0; i < N; i++) {
        stencil st;
        int e = make_stencil(pts + 3 * i, r, &st);
        if (e) return e;
        for (int v = 0; v < 8; v++)
            for (int ch = 0; ch < nch; ch++)
                grid[ch * n + st.idx[v]] += st.w[v] * (vals ? vals[i * nch + ch] : 1.0);
    }
    return ORACLE_OK;
}

int oracle_splat(int r, int64_t N, const double *pts, const double *vals, int nch,
                 double *grid)
{
    if (!is_pow2(r) || N < 0 || nch < 1 || !pts || !grid) return ORACLE_EINVAL;
    return splat(r, N, pts, vals, nch, grid);
}

/* Trilinear lookup of a real grid at the points: out[i] = sum_j w_ij g_j. */
int oracle_gather(int r, int64_t N, const double *pts, const double *grid, double *out)
{
    if (!is_pow2(r) || N < 0 || !pts || !grid || !out) return ORACLE_EINVAL;
    for (int64_t i = 0; i < N; i++) {
        stencil st;
        int e = make_stencil(pts + 3 * i, r, &st);
        if (e) return e;
        double acc = 0.0;
        for (int v = 0; v < 8; v++) acc += st.w[v] * grid[st.idx[v]];
        out[i] = acc;
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Spectral solve (Eq. 3 / Eq. A5-A7).                                       */
/* H_a(k) = g(k) * i u_a / (-2 pi |u|^2), g(k) = exp(-2 sigma^2 |u|^2 / r^2), */
/* with the DC term zero (R5) and the a-th term zero at k_a = r/2 (R6).      */
/* In a box of side lengths L (R13: voxel size L_d / r along axis d, Eq. A1  */
/* with an anisotropic s), u_d = f_d / L_d cycles per unit length for the    */
/* integer frequency f_d, and the Gaussian keeps sigma in grid units along   */
/* every axis: g = exp(-2 sigma^2 sum_d f_d^2 / r^2). The unit cube (L = 1)  */
/* gives the formula above.                                                  */
/* ------------------------------------------------------------------------ */
static double freq(int k, int r) { return k < r / 2 ? (double)k : (double)(k - r); }

static const double kUnitBox[3] = {1.0, 1.0, 1.0};

static cplx spectral_H(int a, const int k[3], int r, double sigma, const double *box)
{
    if (k[0] == 0 && k[1] == 0 && k[2] == 0) return 0.0;
    if (k[a] == r / 2) return 0.0;
    double f2 = 0.0, u2 = 0.0;
    for (int d = 0; d < 3; d++) {
        double f = k[d] == r / 2 ? (double)(r / 2) : freq(k[d], r);
        f2 += f * f;
        u2 += (f / box[d]) * (f / box[d]);
    }
    double g = exp(-2.0 * sigma * sigma * f2 / ((double)r * (double)r));
    return g * (I * (freq(k[a], r) / box[a])) / (-2.0 * kPi * u2);
}

/* The state the backward pass needs from the forward pass. */
typedef struct {
    int r;
    int64_t N;
    double sigma;
    cplx *vhat[3];   /* DFT of the rasterized normal field, per channel */
    double *chip;    /* chi' (Eq. A8) */
    double mu, s;    /* mean of chi' at the points and chi'(0) - mu */
} fwd_state;

static void free_state(fwd_state *S)
{
    for (int a = 0; a < 3; a++) free(S->vhat[a]);
    free(S->chip);
}

/* pts are unit-cube coordinates (c_d / L_d); box holds the lengths L. */
static int forward_core(int r, double sigma, int64_t N, const double *pts,
                        const double *nrm, const double *box, fwd_state *S)
{
    const int64_t n = (int64_t)r * r * r;
    memset(S, 0, sizeof(*S));
    S->r = r;
    S->N = N;
    S->sigma = sigma;
    int e = ORACLE_OK;
    double *v = malloc(sizeof(double) * (size_t)(3 * n));
    cplx *chihat = malloc(sizeof(cplx) * (size_t)n);
    S->chip = malloc(sizeof(double) * (size_t)n);
    for (int a = 0; a < 3; a++) S->vhat[a] = malloc(sizeof(cplx) * (size_t)n);
    if (!v || !chihat || !S->chip || !S->vhat[0] || !S->vhat[1] || !S->vhat[2]) {
        e = ORACLE_ENOMEM;
        goto out;
    }
    /* Point rasterization (Eq. A2), one channel per normal component. */
    e = splat(r, N, pts, nrm, 3, v);
    if (e) goto out;
    /* v~ = FFT(v) (Eq. A3). */
    for (int a = 0; a < 3; a++) {
        for (int64_t j = 0; j < n; j++) S->vhat[a][j] = v[a * n + j];
        e = fft3(S->vhat[a], r, 0);
        if (e) goto out;
    }
    /* chi~ = sum_a H_a v~_a (Eq. 3). */
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; j++) {
        int k[3] = {(int)(j / ((int64_t)r * r)), (int)((j / r) % r), (int)(j % r)};
        cplx acc = 0.0;
        for (int a = 0; a < 3; a++) acc += spectral_H(a, k, r, sigma, box) * S->vhat[a][j];
        chihat[j] = acc;
    }
    /* chi' = Re IFFT(chi~) (Eq. A8, reading R6). */
    e = fft3(chihat, r, 1);
    if (e) goto out;
    for (int64_t j = 0; j < n; j++) S->chip[j] = creal(chihat[j]);
    /* Mean of chi' at the points (Eq. 4, reading R9). */
    {
        double *f = malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
        if (!f) {
            e = ORACLE_ENOMEM;
            goto out;
        }
        e = oracle_gather(r, N, pts, S->chip, f);
        double acc = 0.0;
        for (int64_t i = 0; i < N; i++) acc += f[i];
        free(f);
        if (e) goto out;
        S->mu = acc / (double)N;
    }
    S->s = S->chip[0] - S->mu; /* reading R7 */
    if (!(fabs(S->s) > 0.0) || !isfinite(S->s)) e = ORACLE_EDEGENERATE;
out:
    free(v);
    free(chihat);
    if (e) free_state(S);
    return e;
}

/*
 * Forward pass: chi = m / |s| * (chi' - mu) (Eq. 4).
 * chi (r^3, required), chi_prime (r^3, optional), mu_s (2 doubles: mu, s;
 * optional).
 */
/* Coordinates in a box of side lengths L as unit-cube coordinates c_d / L_d
 * (reading R13; NULL or the unit box: a copy is not needed). */
static double *to_unit(int64_t N, const double *pts, const double *box)
{
    double *u = malloc(sizeof(double) * (size_t)(3 * (N > 0 ? N : 1)));
    if (!u) return NULL;
    for (int64_t i = 0; i < N; i++)
        for (int d = 0; d < 3; d++) u[3 * i + d] = pts[3 * i + d] / box[d];
    return u;
}

static int valid_box(const double *box)
{
    for (int d = 0; d < 3; d++)
        if (!(box[d] > 0.0) || !isfinite(box[d])) return 0;
    return 1;
}

static int forward_box(int r, double sigma, int64_t N, const double *pts, const double *nrm,
                       const double *box, double *chi, double *chi_prime, double *mu_s)
{
    if (!is_pow2(r) || N < 1 || !pts || !nrm || !chi || !(sigma >= 0.0) || !valid_box(box))
        return ORACLE_EINVAL;
    double *upts = to_unit(N, pts, box);
    if (!upts) return ORACLE_ENOMEM;
    fwd_state S;
    int e = forward_core(r, sigma, N, upts, nrm, box, &S);
    free(upts);
    if (e) return e;
    const int64_t n = (int64_t)r * r * r;
    const double alpha = kM / fabs(S.s);
    for (int64_t j = 0; j < n; j++) chi[j] = alpha * (S.chip[j] - S.mu);
    if (chi_prime) memcpy(chi_prime, S.chip, sizeof(double) * (size_t)n);
    if (mu_s) {
        mu_s[0] = S.mu;
        mu_s[1] = S.s;
    }
    free_state(&S);
    return ORACLE_OK;
}

int oracle_dpsr_forward(int r, double sigma, int64_t N, const double *pts,
                        const double *nrm, double *chi, double *chi_prime,
                        double *mu_s)
{
    return forward_box(r, sigma, N, pts, nrm, kUnitBox, chi, chi_prime, mu_s);
}

/* The same in a periodic box [0, L_0) x [0, L_1) x [0, L_2) (reading R13):
 * pts in box coordinates, the grid's voxel size L_d / r along axis d. */
int oracle_dpsr_forward_box(int r, double sigma, int64_t N, const double *pts,
                            const double *nrm, const double *box, double *chi,
                            double *chi_prime, double *mu_s)
{
    if (!box) return ORACLE_EINVAL;
    return forward_box(r, sigma, N, pts, nrm, box, chi, chi_prime, mu_s);
}

/*
 * Backward pass: given dchi = dL/dchi (r^3), return dL/dpoints and
 * dL/dnormals (N x 3 each), the exact reverse-mode derivative of the forward
 * pass above (reading R12).
 *
 *   alpha = m/|s|, S = sum_j dchi_j, D = sum_j dchi_j (chi'_j - mu)
 *   s_bar = -m sign(s) D / s^2, mu_bar = -alpha S - s_bar
 *   G_bar = alpha dchi + s_bar e_0 + (mu_bar / N) W,   W_j = sum_i w_ij
 *   V_bar_a = Re IFFT(conj(H_a) FFT(G_bar))        (adjoint of Eq. 3 / A8)
 *   dnormals_ia = sum_j w_ij V_bar_a[j]            (adjoint of Eq. A2)
 *   dpoints_i = sum_a n_ia d/dc (sum_j w_ij V_bar_a[j])
 *               + (mu_bar / N) d/dc (sum_j w_ij chi'_j)
 */
/* pts in unit-cube coordinates; dpts are derivatives with respect to them
 * (backward_box turns them into derivatives in box coordinates). */
static int backward_impl(int r, double sigma, int64_t N, const double *pts,
                         const double *nrm, const double *box, const double *dchi,
                         double *dpts, double *dnrm, double *dpts_mean)
{
    if (!is_pow2(r) || N < 1 || !pts || !nrm || !dchi || !dpts || !dnrm ||
        !(sigma >= 0.0))
        return ORACLE_EINVAL;
    fwd_state S;
    int e = forward_core(r, sigma, N, pts, nrm, box, &S);
    if (e) return e;
    const int64_t n = (int64_t)r * r * r;
    const double alpha = kM / fabs(S.s);
    double sumS = 0.0, sumD = 0.0;
    for (int64_t j = 0; j < n; j++) {
        sumS += dchi[j];
        sumD += dchi[j] * (S.chip[j] - S.mu);
    }
    const double sgn = S.s > 0 ? 1.0 : -1.0;
    const double s_bar = -kM * sgn * sumD / (S.s * S.s);
    const double mu_bar = -alpha * sumS - s_bar;

    double *W = malloc(sizeof(double) * (size_t)n);
    cplx *Ghat = malloc(sizeof(cplx) * (size_t)n);
    cplx *tmp = malloc(sizeof(cplx) * (size_t)n);
    double *Vbar = malloc(sizeof(double) * (size_t)(3 * n));
    if (!W || !Ghat || !tmp || !Vbar) {
        e = ORACLE_ENOMEM;
        goto out;
    }
    e = splat(r, N, pts, NULL, 1, W);
    if (e) goto out;
    for (int64_t j = 0; j < n; j++) Ghat[j] = alpha * dchi[j] + (mu_bar / (double)N) * W[j];
    Ghat[0] += s_bar;
    e = fft3(Ghat, r, 0);
    if (e) goto out;
    for (int a = 0; a < 3; a++) {
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < n; j++) {
            int k[3] = {(int)(j / ((int64_t)r * r)), (int)((j / r) % r), (int)(j % r)};
            tmp[j] = conj(spectral_H(a, k, r, sigma, box)) * Ghat[j];
        }
        e = fft3(tmp, r, 1);
        if (e) goto out;
        for (int64_t j = 0; j < n; j++) Vbar[a * n + j] = creal(tmp[j]);
    }
    for (int64_t i = 0; i < N; i++) {
        stencil st;
        e = make_stencil(pts + 3 * i, r, &st);
        if (e) goto out;
        double gn[3] = {0, 0, 0}, gc[3] = {0, 0, 0}, gm[3] = {0, 0, 0};
        for (int v = 0; v < 8; v++) {
            for (int a = 0; a < 3; a++) {
                double val = Vbar[a * n + st.idx[v]];
                gn[a] += st.w[v] * val;
                for (int d = 0; d < 3; d++) gc[d] += nrm[3 * i + a] * st.dw[v][d] * val;
            }
            for (int d = 0; d < 3; d++)
                gm[d] += (mu_bar / (double)N) * st.dw[v][d] * S.chip[st.idx[v]];
        }
        for (int d = 0; d < 3; d++) {
            dnrm[3 * i + d] = gn[d];
            dpts[3 * i + d] = gc[d] + gm[d];
            if (dpts_mean) dpts_mean[3 * i + d] = gm[d];
        }
    }
out:
    free(W);
    free(Ghat);
    free(tmp);
    free(Vbar);
    free_state(&S);
    return e;
}

/* The backward pass in a box (reading R13): with x_d = c_d / L_d the unit
 * coordinates the layer works in, dL/dc_d = (1 / L_d) dL/dx_d. */
static int backward_box(int r, double sigma, int64_t N, const double *pts, const double *nrm,
                        const double *box, const double *dchi, double *dpts, double *dnrm,
                        double *dpts_mean)
{
    if (!box || !valid_box(box) || N < 1 || !pts) return ORACLE_EINVAL;
    double *upts = to_unit(N, pts, box);
    if (!upts) return ORACLE_ENOMEM;
    int e = backward_impl(r, sigma, N, upts, nrm, box, dchi, dpts, dnrm, dpts_mean);
    free(upts);
    if (e) return e;
    for (int64_t i = 0; i < N; i++)
        for (int d = 0; d < 3; d++) {
            dpts[3 * i + d] /= box[d];
            if (dpts_mean) dpts_mean[3 * i + d] /= box[d];
        }
    return ORACLE_OK;
}

int oracle_dpsr_backward(int r, double sigma, int64_t N, const double *pts,
                         const double *nrm, const double *dchi, double *dpts,
                         double *dnrm)
{
    return backward_box(r, sigma, N, pts, nrm, kUnitBox, dchi, dpts, dnrm, NULL);
}

int oracle_dpsr_backward_box(int r, double sigma, int64_t N, const double *pts,
                             const double *nrm, const double *box, const double *dchi,
                             double *dpts, double *dnrm)
{
    return backward_box(r, sigma, N, pts, nrm, box, dchi, dpts, dnrm, NULL);
}

/* The same backward pass, also returning the part of dL/dpoints that flows
 * through the mean of Eq. 4, (mu_bar / N) d/dc (sum_j w_ij chi'_j), on its
 * own. With few points this part and the rest nearly cancel (moving a lone
 * point translates chi' and its mean together), which bounds the accuracy any
 * FP32 evaluation of their sum can reach. */
int oracle_dpsr_backward_terms(int r, double sigma, int64_t N, const double *pts,
                               const double *nrm, const double *dchi, double *dpts,
                               double *dnrm, double *dpts_mean)
{
    if (!dpts_mean) return ORACLE_EINVAL;
    return backward_box(r, sigma, N, pts, nrm, kUnitBox, dchi, dpts, dnrm, dpts_mean);
}
