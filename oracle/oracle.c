/*
 * FP64 CPU oracle for the 3D Gaussian Splatting rasterization hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path links, loads or calls
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do. It shares no code, header, table or constant generator with the
 * CUDA library.
 *
 * What it computes (the paper's definition of 3DGS, section 3.2):
 *   Eq. 1  x_i = Pi(mu_i), S_i = J_i Sigma_i J_i^T  (EWA projection, J = dPi/dmu)
 *   Eq. 2  w_i(x) = alpha_i exp(-1/2 (x - x_i)^T S_i^-1 (x - x_i))
 *   Eq. 3  C(x) = sum_i w_i prod_{j<i} (1 - w_j) c_i   (front to back, depth order)
 * with Sigma_i = R(r_i) diag(s_i)^2 R(r_i)^T built from scale and quaternion
 * (Algorithm 1, CovFromScaleRot), colour from real spherical harmonics up to
 * degree 3 (section 3.4, "raw RGB or SH"), frustum and opacity culling
 * (Algorithm 1, Preprocess).
 *
 * Readings where the paper is silent (all are parameters or stated conventions):
 *   - s = exp(log_s); opacity = sigmoid(logit); quaternion (w,x,y,z), normalised;
 *     |q| < 1e-12 is read as the identity rotation.
 *   - low-pass dilation: S += dilation * I (default 0.3 px^2).
 *   - J uses x/z and y/z clamped to +-1.3 tan(half FOV).
 *   - culled if z <= near, if opacity < alpha_min, if det(S) <= 0, or if the
 *     conservative tile rectangle is empty.
 *   - per pixel (centre (x+0.5, y+0.5)) a splat contributes when
 *     q = d^T S^-1 d <= q_max (3-sigma ellipse, q_max = 9) and
 *     alpha = min(alpha_max, o exp(-q/2)) >= alpha_min; compositing stops before
 *     the first splat whose T (1 - alpha) < t_stop (that splat is excluded).
 *   - depth order is by the float32 rounding of the view-space depth, ties broken
 *     by Gaussian index.
 *   - colour = max(0, sum_k sh_k Y_k(dir) + 0.5), dir = normalize(mu - camera
 *     centre), real SH with the Condon-Shortley phase, coefficient index l*l+l+m.
 *   - per-model affine transform M_k = [A | b] (Algorithm 1, x_w = M_k [mu; 1];
 *     section 3.4, the transform is applied to the whole model): the mean goes to
 *     A mu + b and the covariance to A Sigma A^T; the SH colour keeps being evaluated
 *     in the model's own frame, i.e. at the view ray mapped back by A^-1
 *     (dir = normalize(A^-1 (x_w - camera centre))), so a rigidly moved asset carries
 *     its view-dependent colour with it. A singular A is rejected.
 *   - pre-packed attributes (Algorithm 1, "Pre-pack"; section 3.4, FP16 layout): a
 *     Gaussian may be given by its mean, its covariance's upper triangle Sigma^(6)
 *     = (xx, xy, xz, yy, yz, zz) and its opacity alpha directly (the values a packed
 *     buffer decodes to) instead of log-scales, quaternion and logit; everything
 *     downstream of Sigma and alpha is the same.
 *
 * Everything is plain loops in double precision; OpenMP parallelises over
 * independent pixels, tiles or Gaussians only (no change of arithmetic order
 * within one output).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI 3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* Camera and options                                                         */
/* ------------------------------------------------------------------------- */

typedef struct {
    double R[9], t[3];          /* world -> camera: p = R mu + t, row-major */
    double fx, fy, cx, cy, near_z;
    int W, H;
} cam_t;

/* cam17 = [R(9), t(3), fx, fy, cx, cy, near] */
static void load_cam(const double* c, int W, int H, cam_t* cam) {
    for (int k = 0; k < 9; ++k) cam->R[k] = c[k];
    for (int k = 0; k < 3; ++k) cam->t[k] = c[9 + k];
    cam->fx = c[12]; cam->fy = c[13]; cam->cx = c[14]; cam->cy = c[15]; cam->near_z = c[16];
    cam->W = W; cam->H = H;
}

typedef struct {
    int tile;
    double dilation, alpha_min, alpha_max, t_stop, q_max;
} opts_t;

/* opts6 = [tile, dilation, alpha_min, alpha_max, t_stop, q_max] */
static void load_opts(const double* o, opts_t* op) {
    op->tile = (int)o[0];
    op->dilation = o[1]; op->alpha_min = o[2]; op->alpha_max = o[3];
    op->t_stop = o[4]; op->q_max = o[5];
}

/* ------------------------------------------------------------------------- */
/* Real spherical harmonics from Legendre polynomials                         */
/* ------------------------------------------------------------------------- */
/*
 * Y_l^m(x,y,z) on the unit sphere, written as a polynomial in (x,y,z):
 *   Y_l^m = N_l^|m| (-1)^|m| P_l^(|m|)(z) * Re((x+iy)^|m|)   for m > 0
 *   Y_l^m = N_l^|m| (-1)^|m| P_l^(|m|)(z) * Im((x+iy)^|m|)   for m < 0
 *   Y_l^0 = N_l^0 P_l(z)
 * where P_l^(k) is the k-th derivative of the Legendre polynomial and
 *   N_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) * (sqrt(2) if m != 0).
 * This is the associated Legendre function with the Condon-Shortley phase,
 * P_l^m(cos t) = (-1)^m sin^m t d^m P_l/dz^m, times cos/sin(m phi), using
 * sin^m t e^{i m phi} = (x + i y)^m.
 */

static double factorial(int n) { double f = 1; for (int k = 2; k <= n; ++k) f *= k; return f; }

/* coefficients of P_l(z), l = 0..3, c[l][k] multiplies z^k (Bonnet recursion) */
static void legendre_table(double c[4][4]) {
    memset(c, 0, sizeof(double) * 16);
    c[0][0] = 1.0;
    c[1][1] = 1.0;
    for (int l = 1; l < 3; ++l)
        for (int k = 0; k <= l + 1; ++k) {
            double a = (k > 0) ? (2.0 * l + 1.0) * c[l][k - 1] : 0.0;
            double b = (double)l * c[l - 1][k];
            c[l + 1][k] = (a - b) / (l + 1.0);
        }
}

/* value of the d-th derivative of sum_k p[k] z^k (degree <= 3) */
static double poly_deriv_eval(const double p[4], int d, double z) {
    double s = 0.0;
    for (int k = d; k < 4; ++k) {
        double coef = p[k];
        for (int j = 0; j < d; ++j) coef *= (double)(k - j);
        s += coef * pow(z, k - d);
    }
    return s;
}

/* (x + i y)^m as (re, im) */
static void cpow_xy(double x, double y, int m, double* re, double* im) {
    double a = 1.0, b = 0.0;
    for (int k = 0; k < m; ++k) { double na = a * x - b * y, nb = a * y + b * x; a = na; b = nb; }
    *re = a; *im = b;
}

/*
 * Evaluate Y_k (k = l*l+l+m, k < (deg+1)^2) at (x,y,z) treated as a point of R^3
 * (the polynomial extension), and optionally the partial derivatives dY/dx, dY/dy,
 * dY/dz of that polynomial. On the unit sphere the values are the real SH.
 */
static void sh_basis(int deg, double x, double y, double z, double* Y, double* dY /* [K][3] or NULL */) {
    double P[4][4];
    legendre_table(P);
    for (int l = 0; l <= deg; ++l)
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            int k = l * l + l + m;
            double N = sqrt((2.0 * l + 1.0) / (4.0 * PI) * factorial(l - am) / factorial(l + am));
            if (m != 0) N *= sqrt(2.0);
            double sgn = (am % 2) ? -1.0 : 1.0;
            double Pz = poly_deriv_eval(P[l], am, z);
            double re, im;
            cpow_xy(x, y, am, &re, &im);
            double tr = (m >= 0) ? re : im;
            Y[k] = N * sgn * Pz * tr;
            if (dY) {
                double dPz = poly_deriv_eval(P[l], am + 1, z);
                /* d/dx (x+iy)^am = am (x+iy)^(am-1);  d/dy = i am (x+iy)^(am-1) */
                double re1 = 0, im1 = 0;
                if (am > 0) cpow_xy(x, y, am - 1, &re1, &im1);
                double dx_re = am * re1, dx_im = am * im1;
                double dy_re = -am * im1, dy_im = am * re1;
                double dtr_dx = (m >= 0) ? dx_re : dx_im;
                double dtr_dy = (m >= 0) ? dy_re : dy_im;
                dY[k * 3 + 0] = N * sgn * Pz * dtr_dx;
                dY[k * 3 + 1] = N * sgn * Pz * dtr_dy;
                dY[k * 3 + 2] = N * sgn * dPz * tr;
            }
        }
}

/* Exported for the SH pins: Y[(deg+1)^2] at a unit direction. */
void orc_sh_eval(int deg, double x, double y, double z, double* Y) { sh_basis(deg, x, y, z, Y, NULL); }

/* ------------------------------------------------------------------------- */
/* Covariance (Algorithm 1, CovFromScaleRot)                                   */
/* ------------------------------------------------------------------------- */

static void quat_to_rot(const double q_in[4], double R[9]) {
    double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = 1, x = 0, y = 0, z = 0;
    if (n >= 1e-12) { w = q_in[0] / n; x = q_in[1] / n; y = q_in[2] / n; z = q_in[3] / n; }
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Sigma = R diag(s)^2 R^T, full 3x3 row-major */
static void covariance3d(const double* log_s, const double* quat, double Sig[9]) {
    double q[4] = {quat[0], quat[1], quat[2], quat[3]};
    double R[9];
    quat_to_rot(q, R);
    double s2[3];
    for (int k = 0; k < 3; ++k) { double s = exp((double)log_s[k]); s2[k] = s * s; }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += R[i * 3 + k] * s2[k] * R[j * 3 + k];
            Sig[i * 3 + j] = acc;
        }
}

void orc_covariance(int64_t n, const double* log_scales, const double* quats, double* out9) {
    for (int64_t i = 0; i < n; ++i) covariance3d(log_scales + 3 * i, quats + 4 * i, out9 + 9 * i);
}

/* ------------------------------------------------------------------------- */
/* Preprocess: per Gaussian projection, conic, extent, colour (Eq. 1, Alg. 1)  */
/* ------------------------------------------------------------------------- */

typedef struct {
    const double *means, *log_scales, *quats, *logits, *sh;
    int deg;
    int64_t n;
    /* per-model affine transform x_w = A mu + b (Algorithm 1, M_k); has_model 0 = identity */
    int has_model;
    double A[9], b[3], Ainv[9];
    /* pre-packed form: covariance upper triangle [n,6] and opacity [n] given directly
     * (NULL: from log_scales, quats and logits) */
    const double *cov6, *opacity;
} scene_t;

/* model-space covariance of Gaussian i: from Sigma^(6) when given, else CovFromScaleRot */
static void model_cov(const scene_t* sc, int64_t i, double Sig[9]) {
    if (sc->cov6) {
        const double* c = sc->cov6 + 6 * i;
        Sig[0] = c[0]; Sig[1] = c[1]; Sig[2] = c[2];
        Sig[3] = c[1]; Sig[4] = c[3]; Sig[5] = c[4];
        Sig[6] = c[2]; Sig[7] = c[4]; Sig[8] = c[5];
        return;
    }
    covariance3d(sc->log_scales + 3 * i, sc->quats + 4 * i, Sig);
}

/* opacity of Gaussian i: given, or sigmoid(logit) */
static double model_opacity(const scene_t* sc, int64_t i) {
    if (sc->opacity) return sc->opacity[i];
    return 1.0 / (1.0 + exp(-(double)sc->logits[i]));
}

/* model12 = [A | b] row-major 3x4, or NULL for the identity. Returns 1 if A is singular
 * or not finite. */
static int load_model(const double* model12, scene_t* sc) {
    sc->has_model = 0;
    if (!model12) return 0;
    for (int k = 0; k < 12; ++k)
        if (!isfinite(model12[k])) return 1;
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) sc->A[r * 3 + c] = model12[r * 4 + c];
        sc->b[r] = model12[r * 4 + 3];
    }
    const double* A = sc->A;
    /* inverse by the adjugate: Ainv = adj(A) / det(A) */
    double adj[9] = {
        A[4] * A[8] - A[5] * A[7], A[2] * A[7] - A[1] * A[8], A[1] * A[5] - A[2] * A[4],
        A[5] * A[6] - A[3] * A[8], A[0] * A[8] - A[2] * A[6], A[2] * A[3] - A[0] * A[5],
        A[3] * A[7] - A[4] * A[6], A[1] * A[6] - A[0] * A[7], A[0] * A[4] - A[1] * A[3]};
    double det = A[0] * adj[0] + A[1] * adj[3] + A[2] * adj[6];
    if (!(fabs(det) > 0.0) || !isfinite(det)) return 1;
    for (int k = 0; k < 9; ++k) {
        sc->Ainv[k] = adj[k] / det;
        if (!isfinite(sc->Ainv[k])) return 1;
    }
    sc->has_model = 1;
    return 0;
}

/* world-space mean x_w = A mu + b */
static void world_mean(const scene_t* sc, const double* mu, double xw[3]) {
    if (!sc->has_model) { xw[0] = mu[0]; xw[1] = mu[1]; xw[2] = mu[2]; return; }
    for (int r = 0; r < 3; ++r)
        xw[r] = sc->A[r * 3 + 0] * mu[0] + sc->A[r * 3 + 1] * mu[1] + sc->A[r * 3 + 2] * mu[2] + sc->b[r];
}

/* world-space covariance Sigma_w = A Sigma A^T (full 3x3 row-major) */
static void world_cov(const scene_t* sc, const double Sig[9], double Sw[9]) {
    if (!sc->has_model) { memcpy(Sw, Sig, sizeof(double) * 9); return; }
    double AS[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            AS[r * 3 + c] = sc->A[r * 3 + 0] * Sig[0 * 3 + c] + sc->A[r * 3 + 1] * Sig[1 * 3 + c] +
                            sc->A[r * 3 + 2] * Sig[2 * 3 + c];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            Sw[r * 3 + c] = AS[r * 3 + 0] * sc->A[c * 3 + 0] + AS[r * 3 + 1] * sc->A[c * 3 + 1] +
                            AS[r * 3 + 2] * sc->A[c * 3 + 2];
}

/* the SH evaluation ray in the model's own frame (unnormalised): A^-1 (x_w - centre) */
static void model_view_ray(const scene_t* sc, const double xw[3], const double centre[3], double d[3]) {
    double w[3] = {xw[0] - centre[0], xw[1] - centre[1], xw[2] - centre[2]};
    if (!sc->has_model) { d[0] = w[0]; d[1] = w[1]; d[2] = w[2]; return; }
    for (int r = 0; r < 3; ++r)
        d[r] = sc->Ainv[r * 3 + 0] * w[0] + sc->Ainv[r * 3 + 1] * w[1] + sc->Ainv[r * 3 + 2] * w[2];
}

/* Per-Gaussian outputs, all arrays of length n (x2, x3, x4 where noted). */
typedef struct {
    int* valid;          /* 1 if not culled */
    double* uv;          /* [n,2] */
    double* conic;       /* [n,3] a, b, c: q = a dx^2 + 2 b dx dy + c dy^2 */
    double* S;           /* [n,3] s00, s01, s11 (dilated 2D covariance) */
    double* opacity;     /* [n] */
    double* rgb;         /* [n,3] */
    double* z;           /* [n] view depth */
    float* zkey;         /* [n] float32 rounding of z (the sort key) */
    int* radius;         /* [n] */
    int* rect;           /* [n,4] x0, y0, x1, y1 in tiles, upper bounds exclusive */
} prep_t;

static void camera_centre(const cam_t* cam, double c[3]) {
    /* c = -R^T t */
    for (int j = 0; j < 3; ++j)
        c[j] = -(cam->R[0 * 3 + j] * cam->t[0] + cam->R[1 * 3 + j] * cam->t[1] + cam->R[2 * 3 + j] * cam->t[2]);
}

static void preprocess_one(const scene_t* sc, int64_t i, const cam_t* cam, const opts_t* op,
                           int tiles_x, int tiles_y, const prep_t* out) {
    out->valid[i] = 0;
    out->radius[i] = 0;
    for (int k = 0; k < 4; ++k) out->rect[4 * i + k] = 0;
    const double* mu = sc->means + 3 * i;
    double xw[3], p[3];
    world_mean(sc, mu, xw);
    for (int r = 0; r < 3; ++r)
        p[r] = cam->R[r * 3 + 0] * xw[0] + cam->R[r * 3 + 1] * xw[1] + cam->R[r * 3 + 2] * xw[2] + cam->t[r];
    double z = p[2];
    out->z[i] = z;
    out->zkey[i] = (float)z;
    double o = model_opacity(sc, i);
    out->opacity[i] = o;
    if (!(z > cam->near_z)) return;
    if (o < op->alpha_min) return;

    double Sig0[9], Sig[9];
    model_cov(sc, i, Sig0);
    world_cov(sc, Sig0, Sig);

    double limx = 1.3 * (cam->W / (2.0 * cam->fx)), limy = 1.3 * (cam->H / (2.0 * cam->fy));
    double rx = p[0] / z, ry = p[1] / z;
    if (rx > limx) rx = limx;
    if (rx < -limx) rx = -limx;
    if (ry > limy) ry = limy;
    if (ry < -limy) ry = -limy;
    double J[6] = {cam->fx / z, 0.0, -cam->fx * rx / z,
                   0.0, cam->fy / z, -cam->fy * ry / z};
    /* T = J R  (2x3) */
    double T[6];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += J[r * 3 + k] * cam->R[k * 3 + c];
            T[r * 3 + c] = acc;
        }
    /* S = T Sigma T^T + dilation I */
    double S2[4];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
            double acc = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) acc += T[r * 3 + a] * Sig[a * 3 + b] * T[c * 3 + b];
            S2[r * 2 + c] = acc;
        }
    double s00 = S2[0] + op->dilation, s01 = S2[1], s11 = S2[3] + op->dilation;
    double det = s00 * s11 - s01 * s01;
    if (!(det > 0)) return;
    out->S[3 * i + 0] = s00; out->S[3 * i + 1] = s01; out->S[3 * i + 2] = s11;
    out->conic[3 * i + 0] = s11 / det;
    out->conic[3 * i + 1] = -s01 / det;
    out->conic[3 * i + 2] = s00 / det;

    double m = 0.5 * (s00 + s11);
    double disc = m * m - det;
    if (disc < 0.1) disc = 0.1;
    double lam = m + sqrt(disc);
    int rad = (int)ceil(3.0 * sqrt(lam));

    double u = cam->fx * p[0] / z + cam->cx;
    double v = cam->fy * p[1] / z + cam->cy;
    out->uv[2 * i + 0] = u;
    out->uv[2 * i + 1] = v;

    int T_ = op->tile;
    /* clamp in floating point before converting: u, v may be far off screen */
    double fx0 = floor((u - rad - 1.0) / T_), fx1 = floor((u + rad + 1.0) / T_) + 1.0;
    double fy0 = floor((v - rad - 1.0) / T_), fy1 = floor((v + rad + 1.0) / T_) + 1.0;
    int x0 = (int)fmin((double)tiles_x, fmax(0.0, fx0)), x1 = (int)fmin((double)tiles_x, fmax(0.0, fx1));
    int y0 = (int)fmin((double)tiles_y, fmax(0.0, fy0)), y1 = (int)fmin((double)tiles_y, fmax(0.0, fy1));
    out->radius[i] = rad;
    out->rect[4 * i + 0] = x0; out->rect[4 * i + 1] = y0;
    out->rect[4 * i + 2] = x1; out->rect[4 * i + 3] = y1;
    if (x1 <= x0 || y1 <= y0) return;

    /* colour */
    double cc[3], d[3];
    camera_centre(cam, cc);
    model_view_ray(sc, xw, cc, d);
    double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    d[0] /= dn; d[1] /= dn; d[2] /= dn;
    int K = (sc->deg + 1) * (sc->deg + 1);
    double Y[16];
    sh_basis(sc->deg, d[0], d[1], d[2], Y, NULL);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0;
        for (int k = 0; k < K; ++k) acc += (double)sc->sh[((int64_t)i * K + k) * 3 + ch] * Y[k];
        acc += 0.5;
        out->rgb[3 * i + ch] = acc < 0 ? 0.0 : acc;
    }
    out->valid[i] = 1;
}

/* model12: the model's [A | b] (row-major 3x4) or NULL for the identity */
int orc_preprocess(int64_t n, const double* means, const double* log_scales, const double* quats,
                   const double* logits, const double* sh, int deg, const double* model12,
                   const double* cam17, int W, int H, const double* opts6,
                   int* valid, double* uv, double* conic, double* S, double* opacity, double* rgb,
                   double* z, float* zkey, int* radius, int* rect) {
    if (deg < 0 || deg > 3) return 1;
    cam_t cam; load_cam(cam17, W, H, &cam);
    opts_t op; load_opts(opts6, &op);
    scene_t sc;
    memset(&sc, 0, sizeof(sc));
    sc.means = means; sc.log_scales = log_scales; sc.quats = quats; sc.logits = logits; sc.sh = sh;
    sc.deg = deg; sc.n = n;
    if (load_model(model12, &sc)) return 2;
    prep_t out = {valid, uv, conic, S, opacity, rgb, z, zkey, radius, rect};
    int tiles_x = (W + op.tile - 1) / op.tile, tiles_y = (H + op.tile - 1) / op.tile;
    memset(conic, 0, sizeof(double) * 3 * n);
    memset(S, 0, sizeof(double) * 3 * n);
    memset(uv, 0, sizeof(double) * 2 * n);
    memset(rgb, 0, sizeof(double) * 3 * n);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) preprocess_one(&sc, i, &cam, &op, tiles_x, tiles_y, &out);
    return 0;
}

/* The same preprocess for Gaussians given in the pre-packed form: mean, covariance upper
 * triangle cov6 [n,6] = (xx, xy, xz, yy, yz, zz), opacity [n] and SH coefficients. */
int orc_preprocess_cov(int64_t n, const double* means, const double* cov6, const double* opacity,
                       const double* sh, int deg, const double* model12,
                       const double* cam17, int W, int H, const double* opts6,
                       int* valid, double* uv, double* conic, double* S, double* opac_out, double* rgb,
                       double* z, float* zkey, int* radius, int* rect) {
    if (deg < 0 || deg > 3) return 1;
    cam_t cam; load_cam(cam17, W, H, &cam);
    opts_t op; load_opts(opts6, &op);
    scene_t sc;
    memset(&sc, 0, sizeof(sc));
    sc.means = means; sc.sh = sh; sc.deg = deg; sc.n = n; sc.cov6 = cov6; sc.opacity = opacity;
    if (load_model(model12, &sc)) return 2;
    prep_t out = {valid, uv, conic, S, opac_out, rgb, z, zkey, radius, rect};
    int tiles_x = (W + op.tile - 1) / op.tile, tiles_y = (H + op.tile - 1) / op.tile;
    memset(conic, 0, sizeof(double) * 3 * n);
    memset(S, 0, sizeof(double) * 3 * n);
    memset(uv, 0, sizeof(double) * 2 * n);
    memset(rgb, 0, sizeof(double) * 3 * n);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) preprocess_one(&sc, i, &cam, &op, tiles_x, tiles_y, &out);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Compositing one pixel over an ordered candidate list (Eqs. 2-3)            */
/* ------------------------------------------------------------------------- */

typedef struct { float zkey; int64_t idx; } ord_t;

static int cmp_ord(const void* a, const void* b) {
    const ord_t* x = (const ord_t*)a;
    const ord_t* y = (const ord_t*)b;
    if (x->zkey < y->zkey) return -1;
    if (x->zkey > y->zkey) return 1;
    return (x->idx < y->idx) ? -1 : (x->idx > y->idx);
}

/* Ambiguity margins: a decision taken within these of its threshold may go the
 * other way in float32 arithmetic. The float32 renderer evaluates alpha to ~1e-6
 * relative and the transmittance product to ~1e-5 relative after ~100 splats; q
 * carries the rounding of the splat centre relative to the tile centre
 * (|du| * 6e-8 px), which reaches ~2.5e-6 relative at q = 9 for a splat 100 px from
 * the tile centre. Each margin is a safety factor of 8 above that. */
#define AMB_Q_REL     (8.0 * 2.5e-6)
#define AMB_ALPHA_REL (8.0 * 1e-6)
#define AMB_T_REL     (8.0 * 1e-5)
/* the float32 renderer's view depth may differ from zkey (float32 of the FP64 depth) by an ulp */
#define AMB_Z_REL     (8.0 * 1.2e-7)

typedef struct {
    double rgb[3], alpha, T;
    int n_contrib;      /* number of splats composited */
    int last_pos;       /* 1 + position in the ordered list of the last composited splat, 0 if none */
    int ambiguous;
} pix_out_t;

/* Composite pixel centre (pcx, pcy) over `list` (already ordered). zlim: the pixel's depth
 * limit (depth-buffer-aware compositing, a caller-supplied depth buffer tested without
 * writing, section 3.4): a splat whose view depth zkey exceeds it is not composited there
 * (read literally: -infinity rejects every splat, +infinity and NaN none); +infinity when
 * there is no depth buffer. */
static void composite_pixel(const prep_t* pp, const ord_t* list, int64_t len, double pcx, double pcy,
                            double zlim, const double bg[3], const opts_t* op, pix_out_t* out) {
    double T = 1.0, C[3] = {0, 0, 0};
    int n_contrib = 0, last_pos = 0, amb = 0;
    for (int64_t j = 0; j < len; ++j) {
        int64_t i = list[j].idx;
        {
            const double z = (double)list[j].zkey;
            if (isfinite(zlim) && fabs(z - zlim) <= AMB_Z_REL * fabs(zlim)) amb = 1;
            if (z > zlim) continue;   /* a NaN limit compares false: it rejects nothing */
        }
        double dx = pcx - pp->uv[2 * i], dy = pcy - pp->uv[2 * i + 1];
        double a = pp->conic[3 * i], b = pp->conic[3 * i + 1], c = pp->conic[3 * i + 2];
        double q = a * dx * dx + 2.0 * b * dx * dy + c * dy * dy;
        if (fabs(q - op->q_max) <= AMB_Q_REL * op->q_max) {
            /* the cut only matters if the splat would pass the alpha test there */
            if (pp->opacity[i] * exp(-0.5 * q) >= op->alpha_min * (1.0 - AMB_ALPHA_REL)) amb = 1;
        }
        if (q > op->q_max) continue;
        double alpha = pp->opacity[i] * exp(-0.5 * q);
        if (alpha > op->alpha_max) alpha = op->alpha_max;
        if (fabs(alpha - op->alpha_min) <= AMB_ALPHA_REL * op->alpha_min) amb = 1;
        if (alpha < op->alpha_min) continue;
        double Tn = T * (1.0 - alpha);
        if (fabs(Tn - op->t_stop) <= AMB_T_REL * op->t_stop) amb = 1;
        if (Tn < op->t_stop) break;
        for (int ch = 0; ch < 3; ++ch) C[ch] += pp->rgb[3 * i + ch] * alpha * T;
        T = Tn;
        ++n_contrib;
        last_pos = (int)(j + 1);
    }
    for (int ch = 0; ch < 3; ++ch) out->rgb[ch] = C[ch] + T * bg[ch];
    out->alpha = 1.0 - T;
    out->T = T;
    out->n_contrib = n_contrib;
    out->last_pos = last_pos;
    out->ambiguous = amb;
}

static prep_t prep_view(const int* valid, const double* uv, const double* conic, const double* opacity,
                        const double* rgb, const float* zkey) {
    prep_t p;
    memset(&p, 0, sizeof(p));
    p.valid = (int*)valid; p.uv = (double*)uv; p.conic = (double*)conic;
    p.opacity = (double*)opacity; p.rgb = (double*)rgb; p.zkey = (float*)zkey;
    return p;
}

/*
 * Brute force, the plain definition: for each requested pixel, every valid splat
 * is a candidate; candidates are ordered by (zkey, index) and composited.
 * No tiles are involved. px/py: pixel indices; outputs per requested pixel.
 */
int orc_render_pixels(int64_t n, const int* valid, const double* uv, const double* conic,
                      const double* opacity, const double* rgb, const float* zkey,
                      int64_t P, const int* px, const int* py, const double* bg, const double* opts6,
                      const float* zlim /* [P] or NULL */,
                      double* out_rgb, double* out_alpha, double* out_T, int* out_ncontrib,
                      int* out_ambig) {
    opts_t op; load_opts(opts6, &op);
    prep_t pp = prep_view(valid, uv, conic, opacity, rgb, zkey);
    int64_t nv = 0;
    for (int64_t i = 0; i < n; ++i) nv += valid[i] ? 1 : 0;
    ord_t* all = (ord_t*)malloc(sizeof(ord_t) * (nv > 0 ? nv : 1));
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i)
        if (valid[i]) { all[k].zkey = zkey[i]; all[k].idx = i; ++k; }
    qsort(all, nv, sizeof(ord_t), cmp_ord);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < P; ++p) {
        pix_out_t o;
        composite_pixel(&pp, all, nv, px[p] + 0.5, py[p] + 0.5, zlim ? (double)zlim[p] : INFINITY, bg, &op, &o);
        for (int ch = 0; ch < 3; ++ch) out_rgb[3 * p + ch] = o.rgb[ch];
        out_alpha[p] = o.alpha;
        out_T[p] = o.T;
        out_ncontrib[p] = o.n_contrib;
        out_ambig[p] = o.ambiguous;
    }
    free(all);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Tile binning: (tile, depth, index) order, the method's sort order           */
/* ------------------------------------------------------------------------- */

typedef struct {
    int64_t* start;   /* [ntiles + 1] offsets into items */
    ord_t* items;     /* per tile, ordered by (zkey, idx) */
} bins_t;

/* Bin valid splats into the tiles of their rectangles (optionally only tiles with
 * mask[t] != 0), then order each tile's list by (zkey, index). */
static int build_bins(int64_t n, const int* valid, const int* rect, const float* zkey, int tiles_x,
                      int tiles_y, const uint8_t* mask, bins_t* b) {
    int64_t ntiles = (int64_t)tiles_x * tiles_y;
    int64_t* cnt = (int64_t*)calloc(ntiles + 1, sizeof(int64_t));
    if (!cnt) return 1;
    for (int64_t i = 0; i < n; ++i) {
        if (!valid[i]) continue;
        for (int ty = rect[4 * i + 1]; ty < rect[4 * i + 3]; ++ty)
            for (int tx = rect[4 * i + 0]; tx < rect[4 * i + 2]; ++tx) {
                int64_t t = (int64_t)ty * tiles_x + tx;
                if (!mask || mask[t]) cnt[t + 1]++;
            }
    }
    for (int64_t t = 0; t < ntiles; ++t) cnt[t + 1] += cnt[t];
    ord_t* items = (ord_t*)malloc(sizeof(ord_t) * (cnt[ntiles] > 0 ? cnt[ntiles] : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (ntiles > 0 ? ntiles : 1));
    if (!items || !fill) { free(cnt); free(items); free(fill); return 1; }
    for (int64_t t = 0; t < ntiles; ++t) fill[t] = cnt[t];
    for (int64_t i = 0; i < n; ++i) {
        if (!valid[i]) continue;
        for (int ty = rect[4 * i + 1]; ty < rect[4 * i + 3]; ++ty)
            for (int tx = rect[4 * i + 0]; tx < rect[4 * i + 2]; ++tx) {
                int64_t t = (int64_t)ty * tiles_x + tx;
                if (mask && !mask[t]) continue;
                items[fill[t]].zkey = zkey[i];
                items[fill[t]].idx = i;
                fill[t]++;
            }
    }
    free(fill);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < ntiles; ++t)
        qsort(items + cnt[t], cnt[t + 1] - cnt[t], sizeof(ord_t), cmp_ord);
    b->start = cnt;
    b->items = items;
    return 0;
}

static void free_bins(bins_t* b) { free(b->start); free(b->items); }

/*
 * Tile-binned render of the full image (or of the tiles with mask != 0; other
 * pixels are left untouched). Outputs: out_rgb [3,H,W] planar, out_alpha [H,W],
 * out_T [H,W], out_ncontrib [H,W], out_ambig [H,W].
 */
int orc_render_tiled(int64_t n, const int* valid, const double* uv, const double* conic,
                     const double* opacity, const double* rgb, const float* zkey, const int* rect,
                     int W, int H, const double* bg, const double* opts6, const uint8_t* tile_mask,
                     const float* zlim /* [H,W] or NULL */,
                     double* out_rgb, double* out_alpha, double* out_T, int* out_ncontrib,
                     int* out_ambig) {
    opts_t op; load_opts(opts6, &op);
    prep_t pp = prep_view(valid, uv, conic, opacity, rgb, zkey);
    int tiles_x = (W + op.tile - 1) / op.tile, tiles_y = (H + op.tile - 1) / op.tile;
    bins_t b;
    if (build_bins(n, valid, rect, zkey, tiles_x, tiles_y, tile_mask, &b)) return 1;
    int64_t ntiles = (int64_t)tiles_x * tiles_y;
    int64_t HW = (int64_t)H * W;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < ntiles; ++t) {
        if (tile_mask && !tile_mask[t]) continue;
        int tx = (int)(t % tiles_x), ty = (int)(t / tiles_x);
        for (int y = ty * op.tile; y < (ty + 1) * op.tile && y < H; ++y)
            for (int x = tx * op.tile; x < (tx + 1) * op.tile && x < W; ++x) {
                pix_out_t o;
                int64_t pix = (int64_t)y * W + x;
                composite_pixel(&pp, b.items + b.start[t], b.start[t + 1] - b.start[t], x + 0.5, y + 0.5,
                                zlim ? (double)zlim[pix] : INFINITY, bg, &op, &o);
                for (int ch = 0; ch < 3; ++ch) out_rgb[ch * HW + pix] = o.rgb[ch];
                out_alpha[pix] = o.alpha;
                out_T[pix] = o.T;
                out_ncontrib[pix] = o.n_contrib;
                out_ambig[pix] = o.ambiguous;
            }
    }
    free_bins(&b);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Sort-stage oracles: key duplication, stable sort, tile ranges              */
/* ------------------------------------------------------------------------- */

/*
 * Duplicate every valid Gaussian once per tile of its rectangle, in order of
 * Gaussian index then tile (row-major): key = (tile << 32) | bits(zkey), val = i.
 * Returns the number of keys, or -1 if it exceeds cap (nothing past cap written).
 */
int64_t orc_duplicate(int64_t n, const int* valid, const int* rect, const float* zkey, int tiles_x,
                      uint64_t* keys, uint32_t* vals, int64_t cap) {
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!valid[i]) continue;
        uint32_t zb;
        memcpy(&zb, &zkey[i], 4);
        for (int ty = rect[4 * i + 1]; ty < rect[4 * i + 3]; ++ty)
            for (int tx = rect[4 * i + 0]; tx < rect[4 * i + 2]; ++tx) {
                if (m >= cap) return -1;
                uint64_t tile = (uint64_t)ty * (uint64_t)tiles_x + (uint64_t)tx;
                keys[m] = (tile << 32) | (uint64_t)zb;
                vals[m] = (uint32_t)i;
                ++m;
            }
    }
    return m;
}

typedef struct { uint64_t key; int64_t pos; } kp_t;

static int cmp_kp(const void* a, const void* b) {
    const kp_t* x = (const kp_t*)a;
    const kp_t* y = (const kp_t*)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->pos < y->pos) ? -1 : (x->pos > y->pos);
}

/* Stable sort of (keys, vals) by key: equal keys keep their input order. */
int orc_stable_sort_pairs(int64_t m, const uint64_t* keys, const uint32_t* vals, uint64_t* out_keys,
                          uint32_t* out_vals) {
    kp_t* a = (kp_t*)malloc(sizeof(kp_t) * (m > 0 ? m : 1));
    if (!a) return 1;
    for (int64_t j = 0; j < m; ++j) { a[j].key = keys[j]; a[j].pos = j; }
    qsort(a, m, sizeof(kp_t), cmp_kp);
    for (int64_t j = 0; j < m; ++j) { out_keys[j] = a[j].key; out_vals[j] = vals[a[j].pos]; }
    free(a);
    return 0;
}

/* ranges[t] = [start, end) of tile t = key >> 32 in the sorted keys; empty tiles get [0,0). */
int orc_tile_ranges(int64_t m, const uint64_t* sorted_keys, int64_t ntiles, uint32_t* ranges) {
    for (int64_t t = 0; t < ntiles; ++t) { ranges[2 * t] = 0; ranges[2 * t + 1] = 0; }
    int64_t j = 0;
    while (j < m) {
        uint64_t t = sorted_keys[j] >> 32;
        int64_t e = j;
        while (e < m && (sorted_keys[e] >> 32) == t) ++e;
        if ((int64_t)t < ntiles) { ranges[2 * t] = (uint32_t)j; ranges[2 * t + 1] = (uint32_t)e; }
        j = e;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Adjoint (reverse mode of the definition above, decision sets held fixed)   */
/* ------------------------------------------------------------------------- */
/*
 * The paper notes that the splatting formulation is differentiable in all
 * Gaussian parameters (section 3.2, after Eq. 3). This is the FP64 reverse mode
 * of exactly the forward above, for a loss whose gradient with respect to the
 * image is given: gC [3,H,W] (colour) and gA [H,W] (alpha = 1 - T_final).
 *
 * Per pixel, with contributors j = 0..n-1 in depth order, T_j the transmittance
 * before j, T_N the final one and S_j = (sum_{k>j} rgb_k a_k T_k) / T_{j+1}:
 *   dC/drgb_j = a_j T_j
 *   dC/da_j   = T_j (rgb_j - S_j) - T_N bg / (1 - a_j)
 *   dA/da_j   = T_N / (1 - a_j)
 *   S_{j-1}   = rgb_j a_j + (1 - a_j) S_j,   S_{n-1} = 0
 * then a = min(alpha_max, o G), G = exp(-q/2), q = d^T conic d, d = pixel - (u,v).
 * The per-Gaussian screen-space gradients g2 = (u, v, a, b, c, opacity, r, g, b)
 * are then chained through the preprocess: conic = S^-1, S = T Sigma T^T + dil I,
 * T = J R, J(p), p = R x_w + t, x_w = A mu + b, Sigma_w = A Sigma A^T,
 * Sigma = (Rq diag s)(Rq diag s)^T, s = exp(log_s), Rq(q/|q|), opacity = sigmoid(logit),
 * rgb = max(0, sum sh_k Y_k(dir) + 0.5), dir = normalize(A^-1 (x_w - centre)).
 */

typedef struct { int64_t idx; double alpha, T, G, dx, dy; int clamped; } contrib_t;

/* dRq/dqhat_a for a = w, x, y, z (each 3x3 row-major), qhat unit */
static void drot_dq(const double q[4], double dR[4][9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double d[4][9] = {
        /* d/dw */ {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0},
        /* d/dx */ {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x},
        /* d/dy */ {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y},
        /* d/dz */ {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0},
    };
    memcpy(dR, d, sizeof(d));
}

static void preprocess_adjoint_one(const scene_t* sc, int64_t i, const cam_t* cam, const opts_t* op,
                                   const prep_t* pp, const double* g2, double* d_means,
                                   double* d_log_scales, double* d_quats, double* d_logits,
                                   double* d_sh) {
    int K = (sc->deg + 1) * (sc->deg + 1);
    for (int k = 0; k < 3; ++k) { d_means[3 * i + k] = 0; d_log_scales[3 * i + k] = 0; }
    for (int k = 0; k < 4; ++k) d_quats[4 * i + k] = 0;
    d_logits[i] = 0;
    for (int k = 0; k < 3 * K; ++k) d_sh[(int64_t)i * 3 * K + k] = 0;
    if (!pp->valid[i]) return;

    const double* mu = sc->means + 3 * i;
    double gu = g2[0], gv = g2[1], ga = g2[2], gb = g2[3], gc = g2[4], go = g2[5];
    double grgb[3] = {g2[6], g2[7], g2[8]};
    double xw[3], gxw[3] = {0, 0, 0};   /* world-space mean and dL/dx_w */
    world_mean(sc, mu, xw);

    /* colour */
    double cc[3], dv[3];
    camera_centre(cam, cc);
    model_view_ray(sc, xw, cc, dv);
    double dn = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    double dir[3] = {dv[0] / dn, dv[1] / dn, dv[2] / dn};
    double Y[16], dY[48];
    sh_basis(sc->deg, dir[0], dir[1], dir[2], Y, dY);
    double gdir[3] = {0, 0, 0};
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.5;
        for (int k = 0; k < K; ++k) acc += (double)sc->sh[((int64_t)i * K + k) * 3 + ch] * Y[k];
        if (acc < 0) continue;   /* clamped channel: no gradient */
        for (int k = 0; k < K; ++k) {
            d_sh[((int64_t)i * K + k) * 3 + ch] = grgb[ch] * Y[k];
            double c = (double)sc->sh[((int64_t)i * K + k) * 3 + ch];
            for (int a = 0; a < 3; ++a) gdir[a] += grgb[ch] * c * dY[k * 3 + a];
        }
    }
    /* dir = v/|v|: d dir/d v = (I - dir dir^T)/|v|; v = A^-1 (x_w - centre) */
    double dd = gdir[0] * dir[0] + gdir[1] * dir[1] + gdir[2] * dir[2];
    double gv3[3];
    for (int a = 0; a < 3; ++a) gv3[a] = (gdir[a] - dir[a] * dd) / dn;
    for (int a = 0; a < 3; ++a)
        gxw[a] += sc->has_model ? sc->Ainv[0 * 3 + a] * gv3[0] + sc->Ainv[1 * 3 + a] * gv3[1] + sc->Ainv[2 * 3 + a] * gv3[2]
                                : gv3[a];

    /* opacity */
    double o = pp->opacity[i];
    d_logits[i] = go * o * (1.0 - o);

    /* camera-space position */
    double p[3];
    for (int r = 0; r < 3; ++r)
        p[r] = cam->R[r * 3 + 0] * xw[0] + cam->R[r * 3 + 1] * xw[1] + cam->R[r * 3 + 2] * xw[2] + cam->t[r];
    double x = p[0], y = p[1], z = p[2];
    double gp[3] = {0, 0, 0};
    /* u = fx x/z + cx, v = fy y/z + cy */
    gp[0] += gu * cam->fx / z;
    gp[1] += gv * cam->fy / z;
    gp[2] += -gu * cam->fx * x / (z * z) - gv * cam->fy * y / (z * z);

    /* conic = S^-1: dL/dS = -Q Gbar Q with Gbar = [[ga, gb/2], [gb/2, gc]] */
    double Qa = pp->conic[3 * i], Qb = pp->conic[3 * i + 1], Qc = pp->conic[3 * i + 2];
    double Q[4] = {Qa, Qb, Qb, Qc};
    double Gb[4] = {ga, 0.5 * gb, 0.5 * gb, gc};
    double QG[4], MS[4];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) QG[r * 2 + c] = Q[r * 2 + 0] * Gb[0 * 2 + c] + Q[r * 2 + 1] * Gb[1 * 2 + c];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) MS[r * 2 + c] = -(QG[r * 2 + 0] * Q[0 * 2 + c] + QG[r * 2 + 1] * Q[1 * 2 + c]);
    /* MS is the symmetric matrix gradient: dL = tr(MS dS) */

    /* recompute J, T, Sigma */
    double limx = 1.3 * (cam->W / (2.0 * cam->fx)), limy = 1.3 * (cam->H / (2.0 * cam->fy));
    double rx = x / z, ry = y / z;
    int clx = 0, cly = 0;
    if (rx > limx) { rx = limx; clx = 1; } if (rx < -limx) { rx = -limx; clx = 1; }
    if (ry > limy) { ry = limy; cly = 1; } if (ry < -limy) { ry = -limy; cly = 1; }
    double J[6] = {cam->fx / z, 0.0, -cam->fx * rx / z, 0.0, cam->fy / z, -cam->fy * ry / z};
    double T[6];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += J[r * 3 + k] * cam->R[k * 3 + c];
            T[r * 3 + c] = acc;
        }
    double Sig0[9], Sig[9];
    covariance3d(sc->log_scales + 3 * i, sc->quats + 4 * i, Sig0);
    world_cov(sc, Sig0, Sig);

    /* dL/dT = 2 MS T Sigma_w ; dL/dSigma_w = T^T MS T */
    double TS[6];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += T[r * 3 + k] * Sig[k * 3 + c];
            TS[r * 3 + c] = acc;
        }
    double gT[6];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) gT[r * 3 + c] = 2.0 * (MS[r * 2 + 0] * TS[0 * 3 + c] + MS[r * 2 + 1] * TS[1 * 3 + c]);
    double gSigw[9], gSig[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0;
            for (int r = 0; r < 2; ++r)
                for (int c = 0; c < 2; ++c) acc += T[r * 3 + a] * MS[r * 2 + c] * T[c * 3 + b];
            gSigw[a * 3 + b] = acc;
        }
    /* Sigma_w = A Sigma A^T: dL/dSigma = A^T (dL/dSigma_w) A */
    if (sc->has_model) {
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0;
                for (int r = 0; r < 3; ++r)
                    for (int c = 0; c < 3; ++c) acc += sc->A[r * 3 + a] * gSigw[r * 3 + c] * sc->A[c * 3 + b];
                gSig[a * 3 + b] = acc;
            }
    } else {
        memcpy(gSig, gSigw, sizeof(gSig));
    }
    /* T = J R: dL/dJ = dL/dT R^T */
    double gJ[6];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += gT[r * 3 + k] * cam->R[c * 3 + k];
            gJ[r * 3 + c] = acc;
        }
    /* J00 = fx/z, J02 = -fx rx/z, J11 = fy/z, J12 = -fy ry/z, rx = x/z unless clamped */
    gp[2] += gJ[0] * (-cam->fx / (z * z)) + gJ[4] * (-cam->fy / (z * z));
    gp[2] += gJ[2] * (cam->fx * rx / (z * z)) + gJ[5] * (cam->fy * ry / (z * z));
    if (!clx) {
        gp[0] += gJ[2] * (-cam->fx / (z * z));
        gp[2] += gJ[2] * (cam->fx * x / (z * z * z));
    }
    if (!cly) {
        gp[1] += gJ[5] * (-cam->fy / (z * z));
        gp[2] += gJ[5] * (cam->fy * y / (z * z * z));
    }
    /* p = R x_w + t, x_w = A mu + b */
    for (int a = 0; a < 3; ++a)
        gxw[a] += cam->R[0 * 3 + a] * gp[0] + cam->R[1 * 3 + a] * gp[1] + cam->R[2 * 3 + a] * gp[2];
    for (int a = 0; a < 3; ++a)
        d_means[3 * i + a] = sc->has_model
            ? sc->A[0 * 3 + a] * gxw[0] + sc->A[1 * 3 + a] * gxw[1] + sc->A[2 * 3 + a] * gxw[2]
            : gxw[a];

    /* Sigma = M M^T, M = Rq diag(s): dL/dM = 2 gSig M */
    const double* qf = sc->quats + 4 * i;
    double qq[4] = {qf[0], qf[1], qf[2], qf[3]};
    double qn = sqrt(qq[0] * qq[0] + qq[1] * qq[1] + qq[2] * qq[2] + qq[3] * qq[3]);
    double Rq[9];
    quat_to_rot(qq, Rq);
    double s[3];
    for (int k = 0; k < 3; ++k) s[k] = exp((double)sc->log_scales[3 * i + k]);
    double M[9];
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) M[a * 3 + k] = Rq[a * 3 + k] * s[k];
    double gM[9];
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) {
            double acc = 0;
            for (int b = 0; b < 3; ++b) acc += gSig[a * 3 + b] * M[b * 3 + k];
            gM[a * 3 + k] = 2.0 * acc;
        }
    double gs[3] = {0, 0, 0}, gR[9];
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) {
            gs[k] += gM[a * 3 + k] * Rq[a * 3 + k];
            gR[a * 3 + k] = gM[a * 3 + k] * s[k];
        }
    for (int k = 0; k < 3; ++k) d_log_scales[3 * i + k] = gs[k] * s[k];
    if (qn >= 1e-12) {
        double qh[4] = {qq[0] / qn, qq[1] / qn, qq[2] / qn, qq[3] / qn};
        double dR[4][9];
        drot_dq(qh, dR);
        double gqh[4];
        for (int a = 0; a < 4; ++a) {
            double acc = 0;
            for (int e = 0; e < 9; ++e) acc += gR[e] * dR[a][e];
            gqh[a] = acc;
        }
        double dot = gqh[0] * qh[0] + gqh[1] * qh[1] + gqh[2] * qh[2] + gqh[3] * qh[3];
        for (int a = 0; a < 4; ++a) d_quats[4 * i + a] = (gqh[a] - qh[a] * dot) / qn;
    }
}

/* prep arrays for n Gaussians (freed by free_prep) */
static int alloc_prep(int64_t n, prep_t* pp) {
    size_t m = (size_t)(n > 0 ? n : 1);
    pp->valid = (int*)calloc(m, sizeof(int));
    pp->uv = (double*)calloc(2 * m, sizeof(double));
    pp->conic = (double*)calloc(3 * m, sizeof(double));
    pp->S = (double*)calloc(3 * m, sizeof(double));
    pp->opacity = (double*)calloc(m, sizeof(double));
    pp->rgb = (double*)calloc(3 * m, sizeof(double));
    pp->z = (double*)calloc(m, sizeof(double));
    pp->zkey = (float*)calloc(m, sizeof(float));
    pp->radius = (int*)calloc(m, sizeof(int));
    pp->rect = (int*)calloc(4 * m, sizeof(int));
    return !(pp->valid && pp->uv && pp->conic && pp->S && pp->opacity && pp->rgb && pp->z && pp->zkey &&
             pp->radius && pp->rect);
}

static void free_prep(prep_t* pp) {
    free(pp->valid); free(pp->uv); free(pp->conic); free(pp->S); free(pp->opacity); free(pp->rgb);
    free(pp->z); free(pp->zkey); free(pp->radius); free(pp->rect);
}

/* Reverse mode of the compositing (Eqs. 2-3) over the splats of `pp` in the method's
 * (tile, depth, index) order: accumulates the screen-space gradients g2 [n,9] =
 * d/d(u, v, conic a, b, c, opacity, r, g, b). */
static int composite_adjoint(int64_t n, const prep_t* pp_, int W, int H, const opts_t* op_, const double* bg,
                             const double* gC, const double* gA, const float* zlim, double* g2) {
    const prep_t pp = *pp_;
    const opts_t op = *op_;
    int tiles_x = (W + op.tile - 1) / op.tile, tiles_y = (H + op.tile - 1) / op.tile;
    memset(g2, 0, sizeof(double) * 9 * (size_t)n);
    bins_t b;
    if (build_bins(n, pp.valid, pp.rect, pp.zkey, tiles_x, tiles_y, NULL, &b)) return 1;
    int64_t ntiles = (int64_t)tiles_x * tiles_y;
    int64_t HW = (int64_t)H * W;

#pragma omp parallel
    {
        int64_t cap = 256;
        contrib_t* cl = (contrib_t*)malloc(sizeof(contrib_t) * cap);
        double* acc = NULL;
        int64_t acc_cap = 0;
#pragma omp for schedule(dynamic, 1)
        for (int64_t t = 0; t < ntiles; ++t) {
            int64_t len = b.start[t + 1] - b.start[t];
            const ord_t* list = b.items + b.start[t];
            if (len == 0) continue;
            if (len > acc_cap) { free(acc); acc_cap = len; acc = (double*)malloc(sizeof(double) * 9 * acc_cap); }
            memset(acc, 0, sizeof(double) * 9 * len);
            if (len > cap) { free(cl); cap = len; cl = (contrib_t*)malloc(sizeof(contrib_t) * cap); }
            int64_t* posmap = NULL; /* contributor -> list position */
            posmap = (int64_t*)malloc(sizeof(int64_t) * len);
            int tx = (int)(t % tiles_x), ty = (int)(t / tiles_x);
            for (int yy = ty * op.tile; yy < (ty + 1) * op.tile && yy < H; ++yy)
                for (int xx = tx * op.tile; xx < (tx + 1) * op.tile && xx < W; ++xx) {
                    double pcx = xx + 0.5, pcy = yy + 0.5;
                    const double zl = zlim ? (double)zlim[(int64_t)yy * W + xx] : INFINITY;
                    /* forward, recording contributors (the same decisions as composite_pixel) */
                    double T = 1.0;
                    int64_t nc = 0;
                    for (int64_t j = 0; j < len; ++j) {
                        int64_t i = list[j].idx;
                        if ((double)list[j].zkey > zl) continue;
                        double dx = pcx - pp.uv[2 * i], dy = pcy - pp.uv[2 * i + 1];
                        double a = pp.conic[3 * i], bb = pp.conic[3 * i + 1], c = pp.conic[3 * i + 2];
                        double q = a * dx * dx + 2.0 * bb * dx * dy + c * dy * dy;
                        if (q > op.q_max) continue;
                        double G = exp(-0.5 * q);
                        double alpha = pp.opacity[i] * G;
                        int clamped = 0;
                        if (alpha > op.alpha_max) { alpha = op.alpha_max; clamped = 1; }
                        if (alpha < op.alpha_min) continue;
                        double Tn = T * (1.0 - alpha);
                        if (Tn < op.t_stop) break;
                        cl[nc].idx = i; cl[nc].alpha = alpha; cl[nc].T = T; cl[nc].G = G;
                        cl[nc].dx = dx; cl[nc].dy = dy; cl[nc].clamped = clamped;
                        posmap[nc] = j;
                        ++nc;
                        T = Tn;
                    }
                    double TN = T;
                    int64_t pix = (int64_t)yy * W + xx;
                    double gc3[3] = {gC[pix], gC[HW + pix], gC[2 * HW + pix]};
                    double ga1 = gA[pix];
                    double Sx[3] = {0, 0, 0};
                    for (int64_t k = nc - 1; k >= 0; --k) {
                        int64_t i = cl[k].idx;
                        double al = cl[k].alpha, Tk = cl[k].T;
                        double* gi = acc + 9 * posmap[k];
                        double galpha = 0;
                        for (int ch = 0; ch < 3; ++ch) {
                            double col = pp.rgb[3 * i + ch];
                            gi[6 + ch] += gc3[ch] * al * Tk;
                            galpha += gc3[ch] * (Tk * (col - Sx[ch]) - TN * bg[ch] / (1.0 - al));
                        }
                        galpha += ga1 * TN / (1.0 - al);
                        for (int ch = 0; ch < 3; ++ch) Sx[ch] = pp.rgb[3 * i + ch] * al + (1.0 - al) * Sx[ch];
                        if (cl[k].clamped) continue;
                        double o = pp.opacity[i], G = cl[k].G;
                        gi[5] += galpha * G;
                        double gq = galpha * o * G * (-0.5);
                        double dx = cl[k].dx, dy = cl[k].dy;
                        double a = pp.conic[3 * i], bb = pp.conic[3 * i + 1], c = pp.conic[3 * i + 2];
                        gi[2] += gq * dx * dx;
                        gi[3] += gq * 2.0 * dx * dy;
                        gi[4] += gq * dy * dy;
                        /* d = pixel - (u, v): dq/du = -(2 a dx + 2 b dy), dq/dv = -(2 b dx + 2 c dy) */
                        gi[0] += gq * -(2.0 * a * dx + 2.0 * bb * dy);
                        gi[1] += gq * -(2.0 * bb * dx + 2.0 * c * dy);
                    }
                }
            for (int64_t j = 0; j < len; ++j) {
                int64_t i = list[j].idx;
                for (int e = 0; e < 9; ++e) {
                    double v = acc[9 * j + e];
                    if (v != 0.0) {
#pragma omp atomic
                        g2[9 * i + e] += v;
                    }
                }
            }
            free(posmap);
        }
        free(cl);
        free(acc);
    }
    free_bins(&b);
    return 0;
}

/* Reverse mode of the preprocess for one model: g2 [n,9] -> gradients of the model's own
 * parameters (model12 as in orc_preprocess). */
static int preprocess_adjoint(const scene_t* sc, const cam_t* cam, const opts_t* op, int W, int H,
                              const prep_t* pp, const double* g2, double* d_means, double* d_log_scales,
                              double* d_quats, double* d_logits, double* d_sh) {
    (void)W; (void)H;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < sc->n; ++i)
        preprocess_adjoint_one(sc, i, cam, op, pp, g2 + 9 * i, d_means, d_log_scales, d_quats, d_logits, d_sh);
    return 0;
}

/* Exported halves of the adjoint, for a render of several models composited in one
 * global order (Algorithm 1): the compositing adjoint over the concatenated splats ... */
int orc_composite_adjoint(int64_t n, const int* valid, const double* uv, const double* conic,
                          const double* opacity, const double* rgb, const float* zkey, const int* rect,
                          int W, int H, const double* opts6, const double* bg, const double* gC,
                          const double* gA, const float* zlim, double* g2_out) {
    opts_t op; load_opts(opts6, &op);
    prep_t pp;
    memset(&pp, 0, sizeof(pp));
    pp.valid = (int*)valid; pp.uv = (double*)uv; pp.conic = (double*)conic; pp.opacity = (double*)opacity;
    pp.rgb = (double*)rgb; pp.zkey = (float*)zkey; pp.rect = (int*)rect;
    return composite_adjoint(n, &pp, W, H, &op, bg, gC, gA, zlim, g2_out);
}

/* ... and the preprocess adjoint of one model, given its slice of g2. */
int orc_preprocess_adjoint(int64_t n, const double* means, const double* log_scales, const double* quats,
                           const double* logits, const double* sh, int deg, const double* model12,
                           const double* cam17, int W, int H, const double* opts6, const double* g2,
                           double* d_means, double* d_log_scales, double* d_quats, double* d_logits,
                           double* d_sh) {
    if (deg < 0 || deg > 3) return 1;
    cam_t cam; load_cam(cam17, W, H, &cam);
    opts_t op; load_opts(opts6, &op);
    scene_t sc;
    memset(&sc, 0, sizeof(sc));
    sc.means = means; sc.log_scales = log_scales; sc.quats = quats; sc.logits = logits; sc.sh = sh;
    sc.deg = deg; sc.n = n;
    if (load_model(model12, &sc)) return 2;
    int tiles_x = (W + op.tile - 1) / op.tile, tiles_y = (H + op.tile - 1) / op.tile;
    prep_t pp;
    if (alloc_prep(n, &pp)) { free_prep(&pp); return 1; }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) preprocess_one(&sc, i, &cam, &op, tiles_x, tiles_y, &pp);
    int rc = preprocess_adjoint(&sc, &cam, &op, W, H, &pp, g2, d_means, d_log_scales, d_quats, d_logits, d_sh);
    free_prep(&pp);
    return rc;
}

/* The whole adjoint of one model's render (model12 as in orc_preprocess). */
int orc_adjoint(int64_t n, const double* means, const double* log_scales, const double* quats,
                const double* logits, const double* sh, int deg, const double* model12, const double* cam17,
                int W, int H, const double* opts6, const double* bg, const double* gC, const double* gA,
                const float* zlim /* [H,W] depth buffer or NULL */,
                double* d_means, double* d_log_scales, double* d_quats, double* d_logits,
                double* d_sh, double* g2_out /* [n,9] or NULL */) {
    if (deg < 0 || deg > 3) return 1;
    cam_t cam; load_cam(cam17, W, H, &cam);
    opts_t op; load_opts(opts6, &op);
    scene_t sc;
    memset(&sc, 0, sizeof(sc));
    sc.means = means; sc.log_scales = log_scales; sc.quats = quats; sc.logits = logits; sc.sh = sh;
    sc.deg = deg; sc.n = n;
    if (load_model(model12, &sc)) return 2;
    int tiles_x = (W + op.tile - 1) / op.tile, tiles_y = (H + op.tile - 1) / op.tile;
    prep_t pp;
    double* g2 = (double*)calloc(9 * (size_t)(n > 0 ? n : 1), sizeof(double));
    if (alloc_prep(n, &pp) || !g2) { free_prep(&pp); free(g2); return 1; }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) preprocess_one(&sc, i, &cam, &op, tiles_x, tiles_y, &pp);
    int rc = composite_adjoint(n, &pp, W, H, &op, bg, gC, gA, zlim, g2);
    if (!rc) rc = preprocess_adjoint(&sc, &cam, &op, W, H, &pp, g2, d_means, d_log_scales, d_quats, d_logits, d_sh);
    if (!rc && g2_out) memcpy(g2_out, g2, sizeof(double) * 9 * (size_t)n);
    free_prep(&pp);
    free(g2);
    return rc;
}
