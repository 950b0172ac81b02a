/*
 * FP64 CPU oracle for edge-illumination (EI) iterative tomography — the
 * linear operators.  TEST INFRASTRUCTURE ONLY: the CUDA library never links,
 * includes or calls this file; only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load it.  It shares no code with the GPU path.
 *
 * Everything here is a plain, slow loop written for checking by eye.
 *
 * Geometry (the paper leaves the discretisation open; these are the readings
 * used throughout):
 *   voxel (r, c) of an n x n slice sits at
 *       x = (c - (n-1)/2) * pitch,   y = ((n-1)/2 - r) * pitch;
 *   detector pixel j of n_det sits at  t_j = (j - (n_det-1)/2) * pitch;
 *   the parallel-beam line of angle theta through t is {x cos(theta) + y sin(theta) = t}.
 *
 * Radon transform R (Eq. 1, the line integral), computed as the paper's
 * "Algorithmic improvements" section describes it — linear interpolation with
 * the indices computed on the fly — in its ray-driven form: the line is
 * sampled once per voxel row when |cos theta| >= |sin theta| (else once per
 * voxel column), each sample is the linear interpolation of the two voxels it
 * falls between, and each sample carries the path length per row (column),
 * pitch / max(|cos theta|, |sin theta|).  Voxels outside the slice are zero.
 *
 * As a matrix, with u = (c - (n-1)/2) cos th + ((n-1)/2 - r) sin th + (n_det-1)/2
 * the detector coordinate of voxel (r, c) in pixel units and
 * ch = max(|cos th|, |sin th|):
 *       R[(a, j), (r, c)] = (pitch / ch) * hat((u - j) / ch),
 *       hat(v) = max(0, 1 - |v|),
 * so a voxel touches at most the two pixels floor(u) and floor(u) + 1.
 * eio_project follows the ray-driven description, eio_backproject the matrix
 * form; the tests check that the two are transposes of each other.
 *
 * D is the finite difference along t that the paper uses for the detector
 * derivative in Eq. 2 / Eq. 4 ("Experimental improvements" section):
 * central in the interior, one-sided at the two ends.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>

static double hat(double v)
{
    double a = fabs(v);
    return a < 1.0 ? 1.0 - a : 0.0;
}

static double voxel(const double *x, int n, int r, int c)
{
    return (r >= 0 && r < n && c >= 0 && c < n) ? x[(size_t)r * n + c] : 0.0;
}

/*
 * p[a][j] = R[x](t_j, theta_a)   (Eq. 1)
 * x: [n][n] row-major; theta: [n_theta] rad; p: [n_theta][n_det].
 */
void eio_project(int n, int n_theta, int n_det, double pitch,
                 const double *theta, const double *x, double *p)
{
    double hn = 0.5 * (n - 1), hd = 0.5 * (n_det - 1);
    #pragma omp parallel for schedule(dynamic)
    for (int a = 0; a < n_theta; ++a) {
        double ct = cos(theta[a]), st = sin(theta[a]);
        for (int j = 0; j < n_det; ++j) {
            double t = j - hd;                  /* pixel units */
            double acc = 0.0;
            if (fabs(ct) >= fabs(st)) {
                /* one sample per row r: the line crosses y = hn - r at
                   x = (t - y sin) / cos, i.e. at column cs */
                for (int r = 0; r < n; ++r) {
                    double cs = (t - (hn - r) * st) / ct + hn;
                    int c0 = (int)floor(cs);
                    double f = cs - c0;
                    acc += (1.0 - f) * voxel(x, n, r, c0) + f * voxel(x, n, r, c0 + 1);
                }
                acc *= pitch / fabs(ct);
            } else {
                /* one sample per column c: the line crosses x = c - hn at
                   y = (t - x cos) / sin, i.e. at row rs */
                for (int c = 0; c < n; ++c) {
                    double rs = hn - (t - (c - hn) * ct) / st;
                    int r0 = (int)floor(rs);
                    double f = rs - r0;
                    acc += (1.0 - f) * voxel(x, n, r0, c) + f * voxel(x, n, r0 + 1, c);
                }
                acc *= pitch / fabs(st);
            }
            p[(size_t)a * n_det + j] = acc;
        }
    }
}

/*
 * x[r][c] = sum_{a,j} R[(a,j),(r,c)] g[a][j]   (the transpose of R)
 * g: [n_theta][n_det]; x: [n][n].  Voxel by voxel, from the matrix form.
 */
void eio_backproject(int n, int n_theta, int n_det, double pitch,
                     const double *theta, const double *g, double *x)
{
    double hn = 0.5 * (n - 1), hd = 0.5 * (n_det - 1);
    double *cs = (double *)malloc(sizeof(double) * 2 * (size_t)(n_theta > 0 ? n_theta : 1));
    for (int a = 0; a < n_theta; ++a) {
        cs[2 * a] = cos(theta[a]);
        cs[2 * a + 1] = sin(theta[a]);
    }
    #pragma omp parallel for schedule(static)
    for (int r = 0; r < n; ++r) {
        for (int c = 0; c < n; ++c) {
            double acc = 0.0;
            for (int a = 0; a < n_theta; ++a) {
                double ct = cs[2 * a], st = cs[2 * a + 1];
                double ch = fmax(fabs(ct), fabs(st));
                double u = (c - hn) * ct + (hn - r) * st + hd;
                int j0 = (int)floor(u);
                for (int j = j0; j <= j0 + 1; ++j)
                    if (j >= 0 && j < n_det)
                        acc += (pitch / ch) * hat((u - j) / ch) * g[(size_t)a * n_det + j];
            }
            x[(size_t)r * n + c] = acc;
        }
    }
    free(cs);
}

/*
 * dp = D p along the detector axis, per angle row (finite differences, used
 * for the refraction term d/dt R[delta] of Eq. 2).
 *   interior:  (p[j+1] - p[j-1]) / (2 pitch)
 *   ends:      (p[1] - p[0]) / pitch,  (p[n-1] - p[n-2]) / pitch
 *   n_det == 1: 0.
 */
void eio_deriv(int n_rows, int n_det, double pitch, const double *p, double *dp)
{
    for (int a = 0; a < n_rows; ++a) {
        const double *q = p + (size_t)a * n_det;
        double *o = dp + (size_t)a * n_det;
        for (int j = 0; j < n_det; ++j) {
            if (n_det == 1)
                o[j] = 0.0;
            else if (j == 0)
                o[j] = (q[1] - q[0]) / pitch;
            else if (j == n_det - 1)
                o[j] = (q[n_det - 1] - q[n_det - 2]) / pitch;
            else
                o[j] = (q[j + 1] - q[j - 1]) / (2.0 * pitch);
        }
    }
}

/*
 * out = D^T g, written out row by row of D (each row k of D scatters g[k]
 * into the columns it touches).
 */
void eio_deriv_T(int n_rows, int n_det, double pitch, const double *g, double *out)
{
    for (int a = 0; a < n_rows; ++a) {
        const double *q = g + (size_t)a * n_det;
        double *o = out + (size_t)a * n_det;
        for (int j = 0; j < n_det; ++j)
            o[j] = 0.0;
        if (n_det == 1)
            continue;
        for (int k = 0; k < n_det; ++k) {
            if (k == 0) {
                o[0] -= q[0] / pitch;
                o[1] += q[0] / pitch;
            } else if (k == n_det - 1) {
                o[n_det - 2] -= q[k] / pitch;
                o[n_det - 1] += q[k] / pitch;
            } else {
                o[k - 1] -= q[k] / (2.0 * pitch);
                o[k + 1] += q[k] / (2.0 * pitch);
            }
        }
    }
}

/* Number of OpenMP threads the loops above use (1 without OpenMP). */
#ifdef _OPENMP
#include <omp.h>
int eio_num_threads(void) { return omp_get_max_threads(); }
void eio_set_num_threads(int t) { omp_set_num_threads(t); }
#else
int eio_num_threads(void) { return 1; }
void eio_set_num_threads(int t) { (void)t; }
#endif
