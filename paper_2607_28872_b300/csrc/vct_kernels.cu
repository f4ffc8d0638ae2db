// CUDA kernels of the VCT + SPH(2) step for sm_103a.
//
// One thread per particle over the cell-sorted SoA.  Neighbour sums are
// templated on the accumulation type R: double (the FP64 form) or float with
// Kahan compensation (the mixed form); per-particle inversions of B_i and the
// SPH(2) moment matrix M_i are always FP64, as are the pressure-equation
// iterate and residual.  No tensor cores: every sum is a gather over about 20
// (2-D) or 56 (3-D) neighbours.
#include <math.h>
#include <stddef.h>
#include <string.h>

#include <mutex>

#include "vct_internal.cuh"

namespace vct {

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------
template <typename R>
struct Acc {
    R s;
    __device__ __forceinline__ Acc() : s(R(0)) {}
    __device__ __forceinline__ void add(R x) { s += x; }
    __device__ __forceinline__ R val() const { return s; }
};

// Kahan (compensated) summation for the FP32 sums of the mixed form.
template <>
struct Acc<float> {
    float s, c;
    __device__ __forceinline__ Acc() : s(0.f), c(0.f) {}
    __device__ __forceinline__ void add(float x)
    {
        float y = x - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ float val() const { return s; }
};

__device__ __forceinline__ void set_error(int32_t *status, int code, int idx)
{
    if (atomicCAS(status, 0, code) == 0) status[1] = idx;
}

// A step kernel does nothing once an earlier kernel of the same call has
// recorded an error: the state is then invalid, the call returns the error
// and writes nothing back, and later steps queued in the call become no-ops.
__device__ __forceinline__ bool step_failed(const int32_t *status)
{
    return *(const volatile int32_t *)status != 0;
}

// Bottom elevation and derivatives h, h_x, h_y, h_xx, h_yy.
__device__ void bathy(const DevParams &P, double x, double y, double h[5])
{
    double v = P.h0 + P.slope_x * x + P.slope_y * y;
    double hx = P.slope_x, hy = P.slope_y, hxx = 0.0, hyy = 0.0;
    if (P.cos_amp != 0.0) {
        double k = 2.0 * 3.14159265358979323846 / P.cos_len;
        double sn, cs;
        sincos(k * x, &sn, &cs);
        v += P.cos_amp * cs;
        hx -= P.cos_amp * k * sn;
        hxx -= P.cos_amp * k * k * cs;
    }
    for (int g = 0; g < P.n_gauss; ++g) {
        double dx = x - P.gcx[g], dy = y - P.gcy[g], inv_s2 = P.ginv2[g];
        double e = P.gamp[g] * exp(-0.5 * (dx * dx + dy * dy) * inv_s2);
        v += e;
        hx -= e * dx * inv_s2;
        hy -= e * dy * inv_s2;
        hxx += e * (dx * dx * inv_s2 - 1.0) * inv_s2;
        hyy += e * (dy * dy * inv_s2 - 1.0) * inv_s2;
    }
    h[0] = v; h[1] = hx; h[2] = hy; h[3] = hxx; h[4] = hyy;
}

// Projected height and metric of Eqs. (VCT), (jacobi), (lap_VCT) for the map
// kinds of Sec. 2.2.
__device__ void map_metric(const DevParams &P, double x, double y, double z, double &zh,
                           double &J, double &sx, double &sy, double &c0, double &c3)
{
    double a = 1.0, ax = 0, ay = 0, axx = 0, ayy = 0, b = 0, bx = 0, by = 0, bxx = 0, byy = 0;
    if (P.kind == VCT_MAP_E) {
        a = P.aspect;
    } else {
        double h[5];
        bathy(P, x, y, h);
        b = -h[0]; bx = -h[1]; by = -h[2]; bxx = -h[3]; byy = -h[4];
        if (P.kind == VCT_MAP_BFE) {
            a = P.aspect;
        } else if (P.kind == VCT_MAP_SIGMA) {
            double D = P.H - h[0];
            if (D <= 0.0) {
                a = P.amax;
            } else {
                double ai = P.H_hat / D;
                if (ai < P.amin) a = P.amin;
                else if (ai > P.amax) a = P.amax;
                else {
                    double iD = 1.0 / D;
                    a = ai;
                    ax = P.H_hat * h[1] * iD * iD;
                    ay = P.H_hat * h[2] * iD * iD;
                    axx = P.H_hat * (h[3] * iD * iD + 2.0 * h[1] * h[1] * iD * iD * iD);
                    ayy = P.H_hat * (h[4] * iD * iD + 2.0 * h[2] * h[2] * iD * iD * iD);
                }
            }
        }
    }
    if (P.dim == 2) {  // a 2-D section has no y direction: h, alpha, beta depend on x only
        ay = ayy = by = byy = 0.0;
    }
    double zeta = z + b;
    zh = a * zeta;
    J = a;
    sx = ax * zeta + a * bx;
    sy = ay * zeta + a * by;
    c0 = (axx + ayy) * zeta + 2.0 * (ax * bx + ay * by) + a * (bxx + byy);
    c3 = a * a + sx * sx + sy * sy;
}

// Cubic spline (Sec. 3.1) and its radial derivative.
template <typename R>
__device__ __forceinline__ void kern_wdw(R r, R inv_l, R ad, R &w, R &dw)
{
    R q = r * inv_l;
    if (q < R(1)) {
        w = ad * (R(1) - R(1.5) * q * q + R(0.75) * q * q * q);
        dw = ad * (R(-3) * q + R(2.25) * q * q) * inv_l;
    } else if (q < R(2)) {
        R t = R(2) - q;
        w = ad * R(0.25) * t * t * t;
        dw = -ad * R(0.75) * t * t * inv_l;
    } else {
        w = R(0);
        dw = R(0);
    }
}

// Second derivative w'' of the cubic spline (FP64; kern_w2t in type T).
template <typename T>
__device__ __forceinline__ T kern_w2t(T r, T inv_l, T ad)
{
    const T q = r * inv_l;
    if (q < T(1)) return ad * (T(-3) + T(4.5) * q) * inv_l * inv_l;
    if (q < T(2)) return ad * T(1.5) * (T(2) - q) * inv_l * inv_l;
    return T(0);
}

__device__ __forceinline__ double kern_w2(double r, double inv_l, double ad)
{
    return kern_w2t<double>(r, inv_l, ad);
}

template <int D>
__device__ __forceinline__ void load_hat(const Part &c, int i, double *x)
{
    x[0] = c.xh[i];
    if (D == 3) x[1] = c.yh[i];
    x[D - 1] = c.zh[i];
}

template <int D>
__device__ __forceinline__ void load_phys(const Part &c, int i, double *x)
{
    x[0] = c.x[i];
    if (D == 3) x[1] = c.y[i];
    x[D - 1] = c.z[i];
}

template <int D>
__device__ __forceinline__ void load_vel(const Part &c, int i, double *v)
{
    v[0] = c.u[i];
    if (D == 3) v[1] = c.v[i];
    v[D - 1] = c.w[i];
}

// Mixed-form pair differences without FP64 arithmetic (which this GPU runs at
// a small fraction of its FP32 rate).  A sorted particle's projected position
// (and velocity, and v*) is kept as two FP32 numbers, hi = fl32(x) and
// lo = fl32(x - hi), so x = hi + lo up to u|lo| <= u^2|x| (u = 2^-24).  Then
// (hi_j - hi_i) + (lo_j - lo_i) is x_j - x_i to within u|x_j - x_i| plus a few
// u^2|x|: hi_j - hi_i is exact when hi_i and hi_j are within a factor two of
// each other (Sterbenz) and otherwise rounded relative to the difference
// itself.  That is as accurate as rounding the FP64 difference to FP32.
__device__ __forceinline__ float4 f4_hilo_split(double x, double y, double z, float4 &lo)
{
    const float hx = (float)x, hy = (float)y, hz = (float)z;
    lo = make_float4((float)(x - (double)hx), (float)(y - (double)hy), (float)(z - (double)hz), 0.f);
    return make_float4(hx, hy, hz, 0.f);
}

template <int D>
__device__ __forceinline__ void hilo_diff(const float4 &hj, const float4 &lj, const float4 &hi,
                                          const float4 &li, float *d)
{
    d[0] = __fsub_rn(hj.x, hi.x) + __fsub_rn(lj.x, li.x);
    if (D == 3) d[1] = __fsub_rn(hj.y, hi.y) + __fsub_rn(lj.y, li.y);
    d[D - 1] = __fsub_rn(hj.z, hi.z) + __fsub_rn(lj.z, li.z);
}

// r_ij in the arithmetic of R: FP64 differences rounded to R (FP64 form), or
// the hi/lo FP32 differences (mixed form).
template <int D, typename R>
__device__ __forceinline__ void pair_r(const Part &c, const Work &W, int j, const double *xi,
                                       const float4 &hi, const float4 &li, R *r)
{
    if constexpr (sizeof(R) == sizeof(float)) {
        float d[D];
        hilo_diff<D>(W.hatf[j], W.hatlo[j], hi, li, d);
#pragma unroll
        for (int K = 0; K < D; ++K) r[K] = d[K];
    } else {
        double xj[3];
        load_hat<D>(c, j, xj);
#pragma unroll
        for (int K = 0; K < D; ++K) r[K] = (R)(xj[K] - xi[K]);
    }
}

template <int D, typename R>
__device__ __forceinline__ void qvec(const R *r, R *q)
{
    if (D == 2) {
        q[0] = r[0] * r[0]; q[1] = r[1] * r[1]; q[2] = r[0] * r[1];
    } else {
        q[0] = r[0] * r[0]; q[1] = r[1] * r[1]; q[2] = r[2] * r[2];
        q[3] = r[0] * r[1]; q[4] = r[1] * r[2]; q[5] = r[2] * r[0];
    }
}

// Weights k_a(r) of the 0th-order second derivatives of Espanol & Revenga
// (Eq. sec_0th), in the order of the SPH(2) output D (cross entries doubled):
//   d2 phi/dx^I dx^J ~ sum_j V_j (c r^I r^J/|r|^2 - delta^IJ) (r . grad w)/|r|^2 phi_ij,
// c = d + 2; with grad w = fac r, fac = -w'/|r|, (r . grad w)/|r|^2 = fac.
template <int D, typename R>
__device__ __forceinline__ void er_weights(const R *r, R rr2, R fac, R *k)
{
    const R c = R(D + 2), inv = R(1) / rr2;
    if constexpr (D == 2) {
        k[0] = fac * (c * r[0] * r[0] * inv - R(1));
        k[1] = fac * (c * r[1] * r[1] * inv - R(1));
        k[2] = R(2) * fac * c * r[0] * r[1] * inv;
    } else {
        k[0] = fac * (c * r[0] * r[0] * inv - R(1));
        k[1] = fac * (c * r[1] * r[1] * inv - R(1));
        k[2] = fac * (c * r[2] * r[2] * inv - R(1));
        k[3] = R(2) * fac * c * r[0] * r[1] * inv;
        k[4] = R(2) * fac * c * r[1] * r[2] * inv;
        k[5] = R(2) * fac * c * r[2] * r[0] * inv;
    }
}

// Inverse of a D x D matrix (row-major) by the adjugate.  Returns false if singular.
template <int D>
__device__ bool inv_small(const double *B, double *L)
{
    if (D == 2) {
        double det = B[0] * B[3] - B[1] * B[2];
        double s = fabs(B[0]) + fabs(B[1]) + fabs(B[2]) + fabs(B[3]);
        if (!(fabs(det) > 1e-14 * s * s)) return false;
        double id = 1.0 / det;
        L[0] = B[3] * id; L[1] = -B[1] * id; L[2] = -B[2] * id; L[3] = B[0] * id;
        return true;
    } else {
        double c00 = B[4] * B[8] - B[5] * B[7], c01 = B[5] * B[6] - B[3] * B[8], c02 = B[3] * B[7] - B[4] * B[6];
        double det = B[0] * c00 + B[1] * c01 + B[2] * c02;
        double s = 0.0;
        for (int k = 0; k < 9; ++k) s = fmax(s, fabs(B[k]));
        if (!(fabs(det) > 1e-14 * s * s * s)) return false;
        double id = 1.0 / det;
        L[0] = c00 * id;
        L[1] = (B[2] * B[7] - B[1] * B[8]) * id;
        L[2] = (B[1] * B[5] - B[2] * B[4]) * id;
        L[3] = c01 * id;
        L[4] = (B[0] * B[8] - B[2] * B[6]) * id;
        L[5] = (B[2] * B[3] - B[0] * B[5]) * id;
        L[6] = c02 * id;
        L[7] = (B[1] * B[6] - B[0] * B[7]) * id;
        L[8] = (B[0] * B[4] - B[1] * B[3]) * id;
        return true;
    }
}

// Smallest eigenvalue of B_i (over all particle types, symmetrised) below which
// a fluid particle counts as isolated; 1 for a full kernel support, ~0.5 at a
// flat free surface, ~0.1 at a corner of the fluid.
constexpr double LAM_ISOLATED = 0.05;

// Smallest eigenvalue of a symmetric 3 x 3 matrix by cyclic Jacobi rotations
// (each rotation zeroes one off-diagonal entry; the diagonal converges to the
// eigenvalues with an absolute error of a few eps |S|).
__device__ double sym_lam_min_jacobi3(const double *S)
{
    double A[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) A[k] = S[k];
    for (int sweep = 0; sweep < 30; ++sweep) {
        const double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
        const double dia = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
        if (off <= 1e-36 * dia || off < 1e-300) break;
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int q = p + 1; q < 3; ++q) {
                const double apq = A[p * 3 + q];
                if (apq == 0.0) continue;
                const double theta = 0.5 * (A[q * 3 + q] - A[p * 3 + p]) / apq;
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const double akp = A[k * 3 + p], akq = A[k * 3 + q];
                    A[k * 3 + p] = cs * akp - sn * akq;
                    A[k * 3 + q] = sn * akp + cs * akq;
                }
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const double apk = A[p * 3 + k], aqk = A[q * 3 + k];
                    A[p * 3 + k] = cs * apk - sn * aqk;
                    A[q * 3 + k] = sn * apk + cs * aqk;
                }
            }
    }
    return fmin(A[0], fmin(A[4], A[8]));
}

// Smallest eigenvalue of a symmetric D x D matrix: closed form in 2-D; in 3-D
// the trigonometric form of the cubic's roots, except where the two smallest
// eigenvalues cluster (the cosine argument near 1, where acos loses half the
// digits): there cyclic Jacobi rotations.
template <int D>
__device__ double sym_lam_min(const double *S)
{
    if (D == 2) {
        double m = 0.5 * (S[0] + S[3]), h = 0.5 * (S[0] - S[3]);
        return m - sqrt(h * h + S[1] * S[1]);
    } else {
        double p1 = S[1] * S[1] + S[2] * S[2] + S[5] * S[5];
        if (p1 == 0.0) return fmin(S[0], fmin(S[4], S[8]));
        double q = (S[0] + S[4] + S[8]) / 3.0;
        double a = S[0] - q, b = S[4] - q, c = S[8] - q;
        double p2 = a * a + b * b + c * c + 2.0 * p1;
        double p = sqrt(p2 / 6.0);
        double ip = 1.0 / p;
        double B0 = a * ip, B4 = b * ip, B8 = c * ip, B1 = S[1] * ip, B2 = S[2] * ip, B5 = S[5] * ip;
        double det = B0 * (B4 * B8 - B5 * B5) - B1 * (B1 * B8 - B5 * B2) + B2 * (B1 * B5 - B4 * B2);
        double r = fmin(1.0, fmax(-1.0, 0.5 * det));
        if (r > 0.5) return sym_lam_min_jacobi3(S);
        double phi = acos(r) / 3.0;
        return q + 2.0 * p * cos(phi + 2.0 * 3.14159265358979323846 / 3.0);
    }
}

// Gaussian elimination with partial pivoting on an m x m system with nrhs
// right-hand sides (columns of B, row-major m x nrhs).  FP64.
template <int M, int NR>
__device__ bool lu_solve(double *A, double *B)
{
    double amax = 0.0;
#pragma unroll
    for (int k = 0; k < M * M; ++k) amax = fmax(amax, fabs(A[k]));
    if (!(amax > 0.0)) return false;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        int piv = k;
        double pv = fabs(A[k * M + k]);
#pragma unroll
        for (int r = k + 1; r < M; ++r)
            if (fabs(A[r * M + k]) > pv) { pv = fabs(A[r * M + k]); piv = r; }
        if (!(pv > 1e-14 * amax)) return false;
        if (piv != k) {
#pragma unroll
            for (int c = 0; c < M; ++c) {
                double t = A[k * M + c];
                A[k * M + c] = A[piv * M + c];
                A[piv * M + c] = t;
            }
#pragma unroll
            for (int c = 0; c < NR; ++c) {
                double t = B[k * NR + c];
                B[k * NR + c] = B[piv * NR + c];
                B[piv * NR + c] = t;
            }
        }
        double inv = 1.0 / A[k * M + k];
#pragma unroll
        for (int r = k + 1; r < M; ++r) {
            double f = A[r * M + k] * inv;
#pragma unroll
            for (int c = k; c < M; ++c) A[r * M + c] -= f * A[k * M + c];
#pragma unroll
            for (int c = 0; c < NR; ++c) B[r * NR + c] -= f * B[k * NR + c];
        }
    }
#pragma unroll
    for (int k = M - 1; k >= 0; --k) {
#pragma unroll
        for (int c = 0; c < NR; ++c) {
            double s = B[k * NR + c];
#pragma unroll
            for (int j = k + 1; j < M; ++j) s -= A[k * M + j] * B[j * NR + c];
            B[k * NR + c] = s / A[k * M + k];
        }
    }
    return true;
}

// The same elimination kept as factors, for one matrix with two systems
// (M x = B and M^T w = c).  lu_factor runs lu_solve's elimination on A alone:
// at step k rows k and piv[k] are swapped in the columns not yet eliminated and
// the multipliers are stored below the diagonal where they were formed, so
// lu_apply (swap, then subtract, step by step) repeats lu_solve's operations on
// B exactly.  For M^T: M = P_0 E_0^-1 ... P_(m-1) E_(m-1)^-1 U with E_k the
// step-k row operations, so M^-T c = P_0 E_0^T ... P_(m-1) E_(m-1)^T U^-T c.
template <int M>
__device__ bool lu_factor(double *A, int *piv)
{
    double amax = 0.0;
#pragma unroll
    for (int k = 0; k < M * M; ++k) amax = fmax(amax, fabs(A[k]));
    bool ok = amax > 0.0;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        int p = k;
        double pv = fabs(A[k * M + k]);
#pragma unroll
        for (int r = k + 1; r < M; ++r)
            if (fabs(A[r * M + k]) > pv) { pv = fabs(A[r * M + k]); p = r; }
        if (!(pv > 1e-14 * amax)) ok = false;
        piv[k] = p;
        if (p != k) {
#pragma unroll
            for (int c = k; c < M; ++c) {
                double t = A[k * M + c];
                A[k * M + c] = A[p * M + c];
                A[p * M + c] = t;
            }
        }
        double inv = 1.0 / A[k * M + k];
#pragma unroll
        for (int r = k + 1; r < M; ++r) {
            double f = A[r * M + k] * inv;
            A[r * M + k] = f;
#pragma unroll
            for (int c = k + 1; c < M; ++c) A[r * M + c] -= f * A[k * M + c];
        }
    }
    return ok;
}

template <int M, int NR>
__device__ void lu_apply(const double *A, const int *piv, double *B)
{
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const int p = piv[k];
        if (p != k) {
#pragma unroll
            for (int c = 0; c < NR; ++c) {
                double t = B[k * NR + c];
                B[k * NR + c] = B[p * NR + c];
                B[p * NR + c] = t;
            }
        }
#pragma unroll
        for (int r = k + 1; r < M; ++r)
#pragma unroll
            for (int c = 0; c < NR; ++c) B[r * NR + c] -= A[r * M + k] * B[k * NR + c];
    }
#pragma unroll
    for (int k = M - 1; k >= 0; --k) {
#pragma unroll
        for (int c = 0; c < NR; ++c) {
            double s = B[k * NR + c];
#pragma unroll
            for (int j = k + 1; j < M; ++j) s -= A[k * M + j] * B[j * NR + c];
            B[k * NR + c] = s / A[k * M + k];
        }
    }
}

template <int M>
__device__ void lu_apply_t(const double *A, const int *piv, double *w)
{
#pragma unroll
    for (int k = 0; k < M; ++k) {   // U^T y = c
        double s = w[k];
#pragma unroll
        for (int j = 0; j < k; ++j) s -= A[j * M + k] * w[j];
        w[k] = s / A[k * M + k];
    }
#pragma unroll
    for (int k = M - 1; k >= 0; --k) {   // E_k^T, then P_k
        double s = w[k];
#pragma unroll
        for (int r = k + 1; r < M; ++r) s -= A[r * M + k] * w[r];
        w[k] = s;
        const int p = piv[k];
        if (p != k) {
            const double t = w[k];
            w[k] = w[p];
            w[p] = t;
        }
    }
}

// Coefficients of the SPH(2) output (cross terms doubled) in c_trans . D^:
// 2-D [1, c3, c4/2], 3-D [1, 1, c3, 0, c5/2, c4/2]; c4 = 2 s_x, c5 = 2 s_y.
template <int D>
__device__ __forceinline__ void ctilde(double c3, double sx, double sy, double *ct)
{
    if (D == 2) {
        ct[0] = 1.0; ct[1] = c3; ct[2] = sx;
    } else {
        ct[0] = 1.0; ct[1] = 1.0; ct[2] = c3; ct[3] = 0.0; ct[4] = sy; ct[5] = sx;
    }
}

// Physical = Jacobian x projected gradient (Eq. grad_VCT), rows x, (y), z.
template <int D>
__device__ __forceinline__ void jac_apply(double J, double sx, double sy, const double *gh,
                                          double *g)
{
    if (D == 2) {
        g[0] = gh[0] + sx * gh[1];
        g[1] = J * gh[1];
    } else {
        g[0] = gh[0] + sx * gh[2];
        g[1] = gh[1] + sy * gh[2];
        g[2] = J * gh[2];
    }
}

__device__ __forceinline__ double vol_of(const DevParams &P, const Part &c, int j)
{
    // V_j = V0 J_j / Jbar_j (Sec. 3.6); V0 under Condition A.
    return P.volume_mode == 0 ? P.V0 : P.V0 * c.J[j] / c.jbar[j];
}

// vol_of(P, c, j) rounded to R, as formed once per step (W.vol, W.volf).
template <typename R>
__device__ __forceinline__ R vol_at(const Work &W, int j)
{
    if constexpr (sizeof(R) == sizeof(float)) return W.volf[j];
    else return (R)W.vol[j];
}

// ---------------------------------------------------------------------------
// Load / store between the caller's arrays and the sorted buffers
// ---------------------------------------------------------------------------
__global__ void k_load(DevParams P, Part c, vct_state s, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    c.x[i] = s.x[i];
    c.y[i] = (P.dim == 3 && s.y) ? s.y[i] : 0.0;
    c.z[i] = s.z[i];
    c.u[i] = s.u[i];
    c.v[i] = (P.dim == 3 && s.v) ? s.v[i] : 0.0;
    c.w[i] = s.w[i];
    c.p[i] = s.p[i];
    c.jbar[i] = s.jbar[i];
    c.type[i] = s.type[i];
    c.orig[i] = i;
}

void launch_load(const DevParams &P, Part cur, vct_state s, int64_t n, cudaStream_t st)
{
    k_load<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(P, cur, s, (int)n);
}

__global__ void k_store_w(DevParams P, Part c, vct_state s, int n, const int32_t *status)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || status[0] != 0) return;
    int o = c.orig[i];
    s.x[o] = c.x[i];
    if (P.dim == 3 && s.y) s.y[o] = c.y[i];
    s.z[o] = c.z[i];
    s.u[o] = c.u[i];
    if (P.dim == 3 && s.v) s.v[o] = c.v[i];
    s.w[o] = c.w[i];
    s.p[o] = c.p[i];
    s.jbar[o] = c.jbar[i];
}

// ---------------------------------------------------------------------------
// a1: map + metric + cell key (current order)
// ---------------------------------------------------------------------------
// Cell index along one axis, clamped to the grid before the integer
// conversion; a non-finite coordinate (NaN) goes to cell 0.
__device__ __forceinline__ int cell_coord(const DevParams &P, double xh, int axis)
{
    double f = floor((xh - P.box_lo[axis]) * P.inv_cell_h);
    int c = !(f >= 0.0) ? 0 : (f > (double)(P.nc[axis] - 1) ? P.nc[axis] - 1 : (int)f);
    return c;
}

__device__ __forceinline__ void map_key_body(const DevParams &P, const Part &c, const Work &W, int n, int bid_)
{
    if (step_failed(W.status)) return;
    int i = bid_ * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double zh, J, sx, sy, c0, c3;
    map_metric(P, c.x[i], P.dim == 3 ? c.y[i] : 0.0, c.z[i], zh, J, sx, sy, c0, c3);
    c.xh[i] = c.x[i];
    c.yh[i] = P.dim == 3 ? c.y[i] : 0.0;
    c.zh[i] = zh;
    c.J[i] = J;
    c.sx[i] = sx;
    c.sy[i] = sy;
    c.c0[i] = c0;
    c.c3[i] = c3;
    if (!(c.jbar[i] > 0.0)) c.jbar[i] = J;   // Jbar^0 = J^0
    int cx = cell_coord(P, c.xh[i], 0);
    int cy = P.dim == 3 ? cell_coord(P, c.yh[i], 1) : 0;
    int cz = cell_coord(P, zh, 2);
    int key = (cz * P.nc[1] + cy) * P.nc[0] + cx;
    W.key[i] = key;
    atomicAdd(&W.cell_count[key], 1);
}

__global__ void k_map_key(DevParams P, Part c, Work W, int n)
{
    map_key_body(P, c, W, n, blockIdx.x);
}

void launch_map_key(const DevParams &P, Part cur, Work W, int64_t n, cudaStream_t st)
{
    cudaMemsetAsync(W.cell_count, 0, sizeof(int32_t) * (W.ncell + 1), st);
    k_map_key<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(P, cur, W, (int)n);
}

// ---------------------------------------------------------------------------
// a2: stable counting sort by cell (ties by caller index) + reorder
// ---------------------------------------------------------------------------
// Exclusive scan of int counts, three kernels.  SCAN_B elements per block.
constexpr int SCAN_T = 256, SCAN_V = 4, SCAN_B = SCAN_T * SCAN_V;

template <typename T>
__device__ T block_exclusive_scan(T v, T *sh, T &total)
{
    // Hillis-Steele over SCAN_T thread totals in shared memory
    int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int o = 1; o < SCAN_T; o <<= 1) {
        T a = t >= o ? sh[t - o] : T(0);
        __syncthreads();
        sh[t] += a;
        __syncthreads();
    }
    total = sh[SCAN_T - 1];
    T excl = sh[t] - v;
    __syncthreads();
    return excl;
}

template <typename T>
__device__ __forceinline__ void scan_blocks_body(const int32_t *in, T *out, T *blk, int64_t m, int bid_)
{
    __shared__ T sh[SCAN_T];
    int64_t base = (int64_t)bid_ * SCAN_B + (int64_t)threadIdx.x * SCAN_V;
    T loc[SCAN_V], s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_V; ++k) {
        loc[k] = base + k < m ? (T)in[base + k] : T(0);
        s += loc[k];
    }
    T total;
    T ex = block_exclusive_scan<T>(s, sh, total);
#pragma unroll
    for (int k = 0; k < SCAN_V; ++k) {
        if (base + k < m) out[base + k] = ex;
        ex += loc[k];
    }
    if (threadIdx.x == 0) blk[bid_] = total;
}

template <typename T>
__global__ void k_scan_blocks(const int32_t *in, T *out, T *blk, int64_t m)
{
    scan_blocks_body<T>(in, out, blk, m, blockIdx.x);
}

template <typename T>
__device__ __forceinline__ void scan_tops_body(T *blk, int64_t nb, T *out_end, int64_t m, int bid_)
{
    // one block: exclusive scan of nb block totals (nb <= SCAN_T * 64)
    __shared__ T sh[SCAN_T];
    int per = (int)((nb + SCAN_T - 1) / SCAN_T);
    T loc = 0;
    int64_t b0 = (int64_t)threadIdx.x * per;
    for (int k = 0; k < per; ++k)
        if (b0 + k < nb) loc += blk[b0 + k];
    T total;
    T ex = block_exclusive_scan<T>(loc, sh, total);
    for (int k = 0; k < per; ++k)
        if (b0 + k < nb) {
            T v = blk[b0 + k];
            blk[b0 + k] = ex;
            ex += v;
        }
    if (threadIdx.x == 0) out_end[m] = total;
}

template <typename T>
__global__ void k_scan_tops(T *blk, int64_t nb, T *out_end, int64_t m)
{
    scan_tops_body<T>(blk, nb, out_end, m, blockIdx.x);
}

template <typename T>
__device__ __forceinline__ void scan_add_body(T *out, const T *blk, int64_t m, int bid_)
{
    int64_t i = (int64_t)bid_ * blockDim.x + threadIdx.x;
    if (i < m) out[i] += blk[i / SCAN_B];
}

template <typename T>
__global__ void k_scan_add(T *out, const T *blk, int64_t m)
{
    scan_add_body<T>(out, blk, m, blockIdx.x);
}

// out[0..m] = exclusive scan of in[0..m-1], out[m] = total.
template <typename T>
static void exclusive_scan(const int32_t *in, T *out, T *tmp, int64_t m, cudaStream_t st)
{
    int64_t nb = (m + SCAN_B - 1) / SCAN_B;
    if (nb == 0) nb = 1;
    k_scan_blocks<T><<<(unsigned)nb, SCAN_T, 0, st>>>(in, out, tmp, m);
    k_scan_tops<T><<<1, SCAN_T, 0, st>>>(tmp, nb, out, m);
    k_scan_add<T><<<(unsigned)((m + 255) / 256), 256, 0, st>>>(out, tmp, m);
}

__device__ __forceinline__ void scatter_body(const Work &W, const Part &c, int n, int bid_)
{
    if (step_failed(W.status)) return;
    int i = bid_ * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int key = W.key[i];
    int slot = W.cell_start[key] + atomicAdd(&W.cursor[key], 1);
    W.perm[slot] = i;
}

__global__ void k_scatter(Work W, const Part c, int n)
{
    scatter_body(W, c, n, blockIdx.x);
}

// Within each cell, order particles by caller index (deterministic layout).
__device__ __forceinline__ void cell_sort_body(const Work &W, const Part &c, int64_t ncell, int bid_)
{
    if (step_failed(W.status)) return;
    int64_t cell = (int64_t)bid_ * blockDim.x + threadIdx.x;
    if (cell >= ncell) return;
    int a = W.cell_start[cell], b = W.cell_start[cell + 1];
    for (int k = a + 1; k < b; ++k) {
        int v = W.perm[k];
        int key = c.orig[v];
        int m = k - 1;
        while (m >= a && c.orig[W.perm[m]] > key) {
            W.perm[m + 1] = W.perm[m];
            --m;
        }
        W.perm[m + 1] = v;
    }
}

__global__ void k_cell_sort(Work W, const Part c, int64_t ncell)
{
    cell_sort_body(W, c, ncell, blockIdx.x);
}

__device__ __forceinline__ void reorder_body(const Part &c, const Part &a, const Work &W, int n, const DevParams &P, int bid_)
{
    if (step_failed(W.status)) return;
    int i = bid_ * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int s = W.perm[i];
    a.x[i] = c.x[s]; a.y[i] = c.y[s]; a.z[i] = c.z[s];
    a.u[i] = c.u[s]; a.v[i] = c.v[s]; a.w[i] = c.w[s];
    a.p[i] = c.p[s]; a.jbar[i] = c.jbar[s];
    a.type[i] = c.type[s]; a.orig[i] = c.orig[s];
    a.xh[i] = c.xh[s]; a.yh[i] = c.yh[s]; a.zh[i] = c.zh[s];
    a.J[i] = c.J[s]; a.sx[i] = c.sx[s]; a.sy[i] = c.sy[s]; a.c0[i] = c.c0[s]; a.c3[i] = c.c3[s];
    W.cellid[i] = W.key[s];
    W.jratio[i] = c.J[s] / c.jbar[s];   // J / Jbar, used by every pair of the smoothing
    const bool d3 = P.dim == 3;
    float4 lo;
    W.hatf[i] = f4_hilo_split(c.xh[s], d3 ? c.yh[s] : 0.0, c.zh[s], lo);
    W.hatlo[i] = lo;
    W.velhi[i] = f4_hilo_split(c.u[s], d3 ? c.v[s] : 0.0, c.w[s], lo);
    W.vello[i] = lo;
    const double V = P.volume_mode == 0 ? P.V0 : P.V0 * c.J[s] / c.jbar[s];   // vol_of
    W.vol[i] = V;
    W.volf[i] = (float)V;
}

__global__ void k_reorder(const Part c, Part a, Work W, int n, DevParams P)
{
    reorder_body(c, a, W, n, P, blockIdx.x);
}

void launch_sort(const DevParams &P, Part cur, Part alt, Work W, int64_t n, cudaStream_t st)
{
    exclusive_scan<int32_t>(W.cell_count, W.cell_start, W.scan_tmp, W.ncell, st);
    cudaMemsetAsync(W.cursor, 0, sizeof(int32_t) * W.ncell, st);
    unsigned g = (unsigned)((n + 255) / 256);
    k_scatter<<<g, 256, 0, st>>>(W, cur, (int)n);
    k_cell_sort<<<(unsigned)((W.ncell + 127) / 128), 128, 0, st>>>(W, cur, W.ncell);
    k_reorder<<<g, 256, 0, st>>>(cur, alt, W, (int)n, P);
}

// ---------------------------------------------------------------------------
// a3: neighbour lists (FP64 predicate without FMA, cells in ascending key order)
//
// The predicate |r_ij|^2 < r_e^2 is defined in FP64 (the projected positions'
// differences and squares rounded to nearest, no fused multiply-add).  FP64
// arithmetic runs at a small fraction of the FP32 rate on this GPU, so each
// candidate is first tested in FP32 on the positions rounded to FP32; where
// that value is farther from r_e^2 than its error bound, it decides, and only
// the candidates within the bound are tested in FP64.  The lists are the FP64
// predicate's exactly.
//
// Error bound (u = 2^-24, the unit roundoff of FP32).  With x~ = fl32(x),
// |x~ - x| <= u|x|; the FP32 difference d~ = fl32(x~_j - x~_i) satisfies
// |d~ - d| <= u(|x_i| + |x_j|) + u|d~| (1 + 2u), so, with |x_j| <= |x_i| + |d|,
// |d~ - d| <= e = 2u(|x_i| + |d~|)(1 + 4u).  Over the D coordinates, |sum d~^2 - sum d^2| <=
// sum (2|d~| e + e^2), and summing the squares in FP32 adds at most
// (D + 1)u sum d~^2 <= 4u s~ with s~ the FP32 sum.  The test uses twice that
// bound, which also covers the FP32 roundings of the bound itself and the FP64
// predicate's own roundings (relative 2^-51 at most), against r_e^2 rounded down
// (inside) or up (outside); rounding to nearest is monotone, so fl(s~ + b) <
// re2_dn implies s~ + b < re2_dn in exact arithmetic, and likewise outside.
// Non-finite values fail both tests and go to the FP64 predicate.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float nbr_bound(float ad, float xa)
{
    // one coordinate's share: 2|d~| e + e^2 with e = 2u(|x_i| + |d~|)(1 + 1e-4)
    const float u = 5.9604645e-8f;   // 2^-24
    const float e = 2.0002f * u * (xa + ad);
    return 2.f * ad * e + e * e;
}

template <int D>
__device__ __forceinline__ void neighbours_body(const DevParams &P, const Part &c, const Work &W, int n, int bid_)
{
    if (step_failed(W.status)) return;
    int i = bid_ * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double xi[3];
    load_hat<D>(c, i, xi);
    const float4 fi = W.hatf[i];
    const float axi = fabsf(fi.x) * 1.0001f, ayi = fabsf(fi.y) * 1.0001f, azi = fabsf(fi.z) * 1.0001f;
    const float re2_dn = __double2float_rd(P.re2), re2_up = __double2float_ru(P.re2);
    const float u4 = 4.0004f * 5.9604645e-8f;
    int cx = cell_coord(P, xi[0], 0);
    int cy = D == 3 ? cell_coord(P, xi[1], 1) : 0;
    int cz = cell_coord(P, xi[D - 1], 2);
    int cnt = 0, over = 0;
    const int64_t cap = W.cap;
    for (int dz = -1; dz <= 1; ++dz) {
        int z2 = cz + dz;
        if (z2 < 0 || z2 >= P.nc[2]) continue;
        for (int dy = (D == 3 ? -1 : 0); dy <= (D == 3 ? 1 : 0); ++dy) {
            int y2 = cy + dy;
            if (y2 < 0 || y2 >= P.nc[1]) continue;
            int row = (z2 * P.nc[1] + y2) * P.nc[0];
            int xa = cx > 0 ? cx - 1 : 0, xb = cx + 1 < P.nc[0] ? cx + 1 : P.nc[0] - 1;
            int a = W.cell_start[row + xa], b = W.cell_start[row + xb + 1];
            for (int j = a; j < b; ++j) {
                if (j == i) continue;
                const float4 fj = W.hatf[j];
                const float fx = __fsub_rn(fj.x, fi.x), fz = __fsub_rn(fj.z, fi.z);
                const float ax = fabsf(fx), az = fabsf(fz);
                float s2 = __fadd_rn(__fmul_rn(fx, fx), __fmul_rn(fz, fz));
                float bnd = nbr_bound(ax, axi) + nbr_bound(az, azi);
                if (D == 3) {
                    const float fy = __fsub_rn(fj.y, fi.y), ay = fabsf(fy);
                    s2 = __fadd_rn(s2, __fmul_rn(fy, fy));
                    bnd += nbr_bound(ay, ayi);
                }
                bnd = 2.f * (bnd + u4 * s2);
                bool in;
                if (s2 + bnd < re2_dn) {
                    in = true;
                } else if (s2 - bnd > re2_up) {
                    in = false;
                } else {   // within the bound (or not finite): the FP64 predicate
                    double d2;
                    double dx = __dsub_rn(c.xh[j], xi[0]);
                    double dz2 = __dsub_rn(c.zh[j], xi[D - 1]);
                    if (D == 2) {
                        d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dz2, dz2));
                    } else {
                        double dy2 = __dsub_rn(c.yh[j], xi[1]);
                        d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy2, dy2)),
                                       __dmul_rn(dz2, dz2));
                    }
                    in = d2 < P.re2;
                }
                if (in) {
                    if (cnt < P.max_nbr) W.nbr[(int64_t)cnt * cap + i] = j;
                    else over = 1;
                    ++cnt;
                }
            }
        }
    }
    if (over) {
        set_error(W.status, VCT_ERR_CAPACITY, i);
        cnt = P.max_nbr;
    }
    W.nbr_cnt[i] = cnt;
    if (P.precision == VCT_FP64) {
        // FP64 form: sum neighbours in ascending caller index, the order of the
        // definition, so the only differences to a plain evaluation are roundings
        for (int k = 1; k < cnt; ++k) {
            int v = W.nbr[(int64_t)k * cap + i], key = c.orig[v], m = k - 1;
            while (m >= 0 && c.orig[W.nbr[(int64_t)m * cap + i]] > key) {
                W.nbr[(int64_t)(m + 1) * cap + i] = W.nbr[(int64_t)m * cap + i];
                --m;
            }
            W.nbr[(int64_t)(m + 1) * cap + i] = v;
        }
    }
}

template <int D>
__global__ void k_neighbours(DevParams P, const Part c, Work W, int n)
{
    neighbours_body<D>(P, c, W, n, blockIdx.x);
}

void launch_neighbours(const DevParams &P, Part cur, Work W, int64_t n, cudaStream_t st)
{
    unsigned g = (unsigned)((n + 127) / 128);
    if (P.dim == 2) k_neighbours<2><<<g, 128, 0, st>>>(P, cur, W, (int)n);
    else k_neighbours<3><<<g, 128, 0, st>>>(P, cur, W, (int)n);
}

// CSR export over caller indices, rows sorted by caller index.
__global__ void k_csr_counts(const Part c, Work W, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    W.scan_tmp[c.orig[i]] = W.nbr_cnt[i];
}

__global__ void k_csr_fill(const Part c, Work W, int n, const int64_t *row_ptr, int32_t *col,
                           int64_t col_cap)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t base = row_ptr[c.orig[i]];
    int cnt = W.nbr_cnt[i];
    if (base + cnt > col_cap) return;
    for (int k = 0; k < cnt; ++k) {
        int v = c.orig[W.nbr[(int64_t)k * W.cap + i]];
        int m = k - 1;
        while (m >= 0 && col[base + m] > v) {
            col[base + m + 1] = col[base + m];
            --m;
        }
        col[base + m + 1] = v;
    }
}

// ---------------------------------------------------------------------------
// a10: volume smoothing, simultaneous form of Eq. (VCT_bar_a): every fluid
// pair is applied once from each end, from the values before the sweep.
// ---------------------------------------------------------------------------
template <int D, typename R>
__device__ __forceinline__ void smoothing_body(const DevParams &P, const Part &c, const Work &W, int n, int bid_)
{
    if (step_failed(W.status)) return;
    int i = bid_ * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double jb = c.jbar[i];
    if (c.type[i] != FLUID) {
        W.jbar_tmp[i] = jb;
        return;
    }
    double xi[3];
    load_hat<D>(c, i, xi);
    double ri = W.jratio[i], sum = 0.0;
    int cnt = W.nbr_cnt[i];
    const float4 hfi = W.hatf[i], lfi = W.hatlo[i];
    const float cvf = (float)P.cv, ref = (float)P.re, inv_re = (float)(1.0 / P.re);
    for (int k = 0; k < cnt; ++k) {
        int j = W.nbr[(int64_t)k * W.cap + i];
        if (c.type[j] != FLUID) continue;
        if constexpr (sizeof(R) == sizeof(float)) {
            // mixed: distance and weight in FP32 from the hi/lo positions; the
            // J/Jbar difference (small against J/Jbar itself) and the sum in FP64
            float d[D], rr2 = 0.f;
            hilo_diff<D>(W.hatf[j], W.hatlo[j], hfi, lfi, d);
#pragma unroll
            for (int K = 0; K < D; ++K) rr2 += d[K] * d[K];
            const float wgt = cvf * (ref - sqrtf(rr2)) * inv_re;
            sum += (double)wgt * (W.jratio[j] - ri);
        } else {
            double xj[3], rr2 = 0.0;
            load_hat<D>(c, j, xj);
            for (int K = 0; K < D; ++K) rr2 += (xj[K] - xi[K]) * (xj[K] - xi[K]);
            double rr = sqrt(rr2);
            sum += P.cv * (P.re - rr) / P.re * (W.jratio[j] - ri);
        }
    }
    const double jb_new = c.J[i] / (ri + 2.0 * sum);
    W.jbar_tmp[i] = jb_new;
    const double V = P.V0 * c.J[i] / jb_new;   // vol_of with the smoothed Jbar
    W.vol[i] = V;
    W.volf[i] = (float)V;
}

template <int D, typename R>
__global__ void k_smoothing(DevParams P, const Part c, Work W, int n)
{
    smoothing_body<D, R>(P, c, W, n, blockIdx.x);
}

void launch_smoothing(const DevParams &P, Part cur, Work W, int64_t n, cudaStream_t st)
{
    unsigned g = (unsigned)((n + 127) / 128);
    const bool mixed = P.precision == VCT_MIXED;
    if (P.dim == 2) {
        if (mixed) k_smoothing<2, float><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        else k_smoothing<2, double><<<g, 128, 0, st>>>(P, cur, W, (int)n);
    } else {
        if (mixed) k_smoothing<3, float><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        else k_smoothing<3, double><<<g, 128, 0, st>>>(P, cur, W, (int)n);
    }
    cudaMemcpyAsync(cur.jbar, W.jbar_tmp, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
}

// Blocks of 128 per SM the passes are compiled for (the register budget):
// measured, 3 instead of 1 (<= 168 registers, more spills): pass 1 3-D slice
// 1.76 -> 1.42 ms, 2-D wave 57 -> 61 us; pass 2 3-D 3.50 -> 3.57 ms, 2-D 81 -> 79 us.
template <int D>
constexpr int pass1_min_blocks() { return D == 3 ? 3 : 1; }
template <int D>
constexpr int pass2_min_blocks() { return D == 2 ? 3 : 1; }

// ---------------------------------------------------------------------------
// a4: pass 1 -- B_i and L_i (Eq. gra_1st), <grad^ v>, C~_i, rho^_i,
// free-surface flag, Smagorinsky eddy viscosity (Sec. 3.4).
// ---------------------------------------------------------------------------
template <int D, typename R>
__device__ __forceinline__ void pass1_body(const DevParams &P, const Part &c, const Work &W, int n, int bid_)
{
    if (step_failed(W.status)) return;
    constexpr int M = D == 2 ? 3 : 6;
    int i = bid_ * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (c.type[i] != FLUID) return;
    const int64_t cap = W.cap;
    double xi[3], pi_[3], vi[3];
    load_hat<D>(c, i, xi);
    const float4 hfi = W.hatf[i], lfi = W.hatlo[i];
    load_phys<D>(c, i, pi_);
    load_vel<D>(c, i, vi);
    const float4 vhi = W.velhi[i], vlo = W.vello[i];
    Acc<R> B[D * D], Ball[D * D], nsum[D], Gv[D * D], Gq[D * M], rho;
    double dwall2 = 1e300;
    const R inv_l = (R)P.inv_l, ad = (R)P.ad;
    const int cnt = W.nbr_cnt[i];
    for (int k = 0; k < cnt; ++k) {
        int j = W.nbr[(int64_t)k * cap + i];
        int tj = c.type[j];
        R r[D], rr2 = R(0);
        pair_r<D, R>(c, W, j, xi, hfi, lfi, r);
#pragma unroll
        for (int K = 0; K < D; ++K) rr2 += r[K] * r[K];
        R rr = sqrt(rr2), w, dw;
        kern_wdw<R>(rr, inv_l, ad, w, dw);
        rho.add((R)P.V0 * w);
        if (rr2 == R(0)) continue;
        R gw[D], fac = -dw / rr;
#pragma unroll
        for (int K = 0; K < D; ++K) gw[K] = fac * r[K];
        const R V0 = (R)P.V0;
#pragma unroll
        for (int K = 0; K < D; ++K) {
            nsum[K].add(V0 * gw[K]);
#pragma unroll
            for (int L2 = 0; L2 < D; ++L2) Ball[K * D + L2].add(V0 * gw[K] * r[L2]);
        }
        if (tj == VIRTUAL) continue;
        R Vj = vol_at<R>(W, j);
        R q[M];
        qvec<D, R>(r, q);
#pragma unroll
        for (int K = 0; K < D; ++K) {
            R vg = Vj * gw[K];
#pragma unroll
            for (int L2 = 0; L2 < D; ++L2) B[K * D + L2].add(vg * r[L2]);
#pragma unroll
            for (int a = 0; a < M; ++a) Gq[K * M + a].add(vg * q[a]);
        }
        R vij[D];
        if constexpr (sizeof(R) == sizeof(float)) {   // mixed: hi/lo differences
            if (tj == FLUID || P.slip) {   // a free-slip wall carries its own velocity
                hilo_diff<D>(W.velhi[j], W.vello[j], vhi, vlo, vij);
            } else {
                vij[0] = -(vhi.x + vlo.x);
                if (D == 3) vij[1] = -(vhi.y + vlo.y);
                vij[D - 1] = -(vhi.z + vlo.z);
            }
        } else {
            double vj[3] = {0.0, 0.0, 0.0};
            if (tj == FLUID || P.slip) load_vel<D>(c, j, vj);
#pragma unroll
            for (int cc = 0; cc < D; ++cc) vij[cc] = (R)(vj[cc] - vi[cc]);
        }
#pragma unroll
        for (int cc = 0; cc < D; ++cc) {
#pragma unroll
            for (int K = 0; K < D; ++K) Gv[cc * D + K].add(Vj * vij[cc] * gw[K]);
        }
        if (tj == WALL) {
            double pj[3], d2 = 0.0;
            load_phys<D>(c, j, pj);
#pragma unroll
            for (int K = 0; K < D; ++K) d2 += (pj[K] - pi_[K]) * (pj[K] - pi_[K]);
            dwall2 = fmin(dwall2, d2);
        }
    }
    double rho_hat = P.rho * ((double)rho.val() + P.V0 * P.ad);   // + self term V0 w(0)
    W.rho_hat[i] = rho_hat;
    double Bd[D * D], L[D * D];
#pragma unroll
    for (int k = 0; k < D * D; ++k) Bd[k] = (double)B[k].val();
    bool iso = false;   // isolated: no correction, no derivatives (see below)
    if (!inv_small<D>(Bd, L)) {
        iso = true;
        for (int k = 0; k < D * D; ++k) L[k] = 0.0;
    }
#pragma unroll
    for (int k = 0; k < D * D; ++k) W.L[(int64_t)k * cap + i] = L[k];
    double gv[D * D];
#pragma unroll
    for (int cc = 0; cc < D; ++cc)
#pragma unroll
        for (int K = 0; K < D; ++K) {
            double s = 0.0;
#pragma unroll
            for (int L2 = 0; L2 < D; ++L2) s += L[K * D + L2] * (double)Gv[cc * D + L2].val();
            gv[cc * D + K] = s;
            W.gv[(int64_t)(cc * D + K) * cap + i] = s;
        }
#pragma unroll
    for (int K = 0; K < D; ++K)
#pragma unroll
        for (int a = 0; a < M; ++a) {
            double s = 0.0;
#pragma unroll
            for (int L2 = 0; L2 < D; ++L2) s += L[K * D + L2] * (double)Gq[L2 * M + a].val();
            W.Ct[(int64_t)(K * M + a) * cap + i] = s;
        }
    // free surface: eigenvalue rule on B over all particles, scan cone between thresholds
    double Bs[D * D];
#pragma unroll
    for (int K = 0; K < D; ++K)
#pragma unroll
        for (int L2 = 0; L2 < D; ++L2)
            Bs[K * D + L2] = 0.5 * ((double)Ball[K * D + L2].val() + (double)Ball[L2 * D + K].val());
    double lam = sym_lam_min<D>(Bs);
    W.lam[i] = lam;
    int fs;
    if (lam <= P.lam_lo) fs = 1;
    else if (lam > P.lam_hi) fs = 0;
    else {
        double Ba[D * D], La[D * D], nrm[D], nn = 0.0;
#pragma unroll
        for (int k = 0; k < D * D; ++k) Ba[k] = (double)Ball[k].val();
        if (!inv_small<D>(Ba, La)) fs = 1;
        else {
#pragma unroll
            for (int K = 0; K < D; ++K) {
                double s = 0.0;
#pragma unroll
                for (int L2 = 0; L2 < D; ++L2) s += La[K * D + L2] * (double)nsum[L2].val();
                nrm[K] = -s;
                nn += s * s;
            }
            nn = sqrt(nn);
            if (!(nn > 0.0)) fs = 0;
            else {
                double T[D], h = P.l, c45 = sqrt(0.5), rlim = sqrt(2.0) * h;
#pragma unroll
                for (int K = 0; K < D; ++K) {
                    nrm[K] /= nn;
                    T[K] = xi[K] + h * nrm[K];
                }
                fs = 1;
                for (int k = 0; k < cnt && fs; ++k) {
                    int j = W.nbr[(int64_t)k * cap + i];
                    double xj[3], rr2 = 0.0, tt2 = 0.0, nr = 0.0;
                    load_hat<D>(c, j, xj);
#pragma unroll
                    for (int K = 0; K < D; ++K) {
                        double rk = xj[K] - xi[K], tk = xj[K] - T[K];
                        rr2 += rk * rk;
                        tt2 += tk * tk;
                        nr += nrm[K] * rk;
                    }
                    double rr = sqrt(rr2);
                    if (rr == 0.0) continue;
                    if (rr >= rlim) {
                        if (sqrt(tt2) < h) fs = 0;
                    } else if (nr > c45 * rr) {
                        fs = 0;
                    }
                }
            }
        }
    }
    // An isolated particle (a splash or droplet: B_i not invertible, or the
    // smallest eigenvalue of B over all particle types below LAM_ISOLATED) is a
    // free-surface particle without corrected derivatives: L_i = 0, so its
    // gradients, SPH(2) second derivatives and pressure gradient vanish and it
    // moves under gravity alone until it has neighbours again.  Flag value 2.
    if (!iso && lam < LAM_ISOLATED) iso = true;
    if (iso) {
#pragma unroll
        for (int k = 0; k < D * D; ++k) {
            W.L[(int64_t)k * cap + i] = 0.0;
            W.gv[(int64_t)k * cap + i] = 0.0;
            gv[k] = 0.0;
        }
#pragma unroll
        for (int k = 0; k < D * M; ++k) W.Ct[(int64_t)k * cap + i] = 0.0;
    }
    W.fs[i] = iso ? 2 : fs;
    // Smagorinsky: nu_E = (C_s f_s r_e)^2 sqrt(2 S:S), S from G = J grad^ v
    double nue = 0.0;
    if (P.smag) {
        double G[D * D];  // G[I*D + cc] = d v_cc / d x_I
#pragma unroll
        for (int cc = 0; cc < D; ++cc) {
            double gh[D], g[D];
#pragma unroll
            for (int K = 0; K < D; ++K) gh[K] = gv[cc * D + K];
            jac_apply<D>(c.J[i], c.sx[i], c.sy[i], gh, g);
#pragma unroll
            for (int I = 0; I < D; ++I) G[I * D + cc] = g[I];
        }
        double SS = 0.0;
#pragma unroll
        for (int I = 0; I < D; ++I)
#pragma unroll
            for (int cc = 0; cc < D; ++cc) {
                double s = 0.5 * (G[I * D + cc] + G[cc * D + I]);
                SS += s * s;
            }
        double fsd = 1.0;
        if (dwall2 < 1e299) fsd = 1.0 - exp(-10.0 * P.d0 / P.ds * sqrt(dwall2) / P.re);
        double cd = P.cs * fsd * P.re;
        nue = cd * cd * sqrt(2.0 * SS);
    }
    W.nu[i] = P.nu_k + nue;
}

template <int D, typename R>
__global__ void __launch_bounds__(128, pass1_min_blocks<D>()) k_pass1(DevParams P, const Part c, Work W, int n)
{
    pass1_body<D, R>(P, c, W, n, blockIdx.x);
}

void launch_pass1(const DevParams &P, Part cur, Work W, int64_t n, cudaStream_t st)
{
    unsigned g = (unsigned)((n + 127) / 128);
    if (P.dim == 2) {
        if (P.precision == VCT_MIXED) k_pass1<2, float><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        else k_pass1<2, double><<<g, 128, 0, st>>>(P, cur, W, (int)n);
    } else {
        if (P.precision == VCT_MIXED) k_pass1<3, float><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        else k_pass1<3, double><<<g, 128, 0, st>>>(P, cur, W, (int)n);
    }
}

// ---------------------------------------------------------------------------
// a5 + a6 + a7 (matrix part): SPH(2) moment matrix M_i (Eq. sec_SPH2), the
// predictor (Eq. VCT_predictor) and the coefficients a_ij of the left side of
// Eq. (VCT_ppe) written as sum_j a_ij (p_j - p_i):
//   a_ij = V_j [ c0 (L grad w_ij)_z + 2 F_ij (w . q_ij) - 2 u . L grad w_ij ],
//   w = M_i^-T c~,  u = sum_j V_j F_ij (w . q_ij) r_ij.
// ---------------------------------------------------------------------------
template <int D, typename R>
__device__ __forceinline__ void pass2_body(const DevParams &P, const Part &c, const Work &W, int n, int predictor, int bid_)
{
    if (step_failed(W.status)) return;
    constexpr int M = D == 2 ? 3 : 6;
    int i = bid_ * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (c.type[i] != FLUID) {
        if (predictor) W.pcnt[i] = -1;
        return;
    }
    const int64_t cap = W.cap;
    double xi[3], vi[3];
    load_hat<D>(c, i, xi);
    const float4 hfi = W.hatf[i], lfi = W.hatlo[i];
    load_vel<D>(c, i, vi);
    R L[D * D], Ct[D * M];
#pragma unroll
    for (int k = 0; k < D * D; ++k) L[k] = (R)W.L[(int64_t)k * cap + i];
#pragma unroll
    for (int k = 0; k < D * M; ++k) Ct[k] = (R)W.Ct[(int64_t)k * cap + i];
    double gvd[D * D];
#pragma unroll
    for (int k = 0; k < D * D; ++k) gvd[k] = W.gv[(int64_t)k * cap + i];
    const double nui = W.nu[i];
    constexpr bool MIXED = sizeof(R) == sizeof(float);
    float gvf[D * D];
#pragma unroll
    for (int k = 0; k < D * D; ++k) gvf[k] = (float)gvd[k];
    const float4 vhi = W.velhi[i], vlo = W.vello[i];
    Acc<R> Mm[M * M], bv[M * D], Gnu[D], Q[M * D];
    const R inv_l = (R)P.inv_l, ad = (R)P.ad;
    const int cnt = W.nbr_cnt[i];
    for (int k = 0; k < cnt; ++k) {
        int j = W.nbr[(int64_t)k * cap + i];
        int tj = c.type[j];
        if (tj == VIRTUAL) continue;
        R r[D], rr2 = R(0);
        double rd[D];
        if constexpr (MIXED) {
            pair_r<D, R>(c, W, j, xi, hfi, lfi, r);
        } else {
            double xj[3];
            load_hat<D>(c, j, xj);
#pragma unroll
            for (int K = 0; K < D; ++K) {
                rd[K] = xj[K] - xi[K];
                r[K] = (R)rd[K];
            }
        }
#pragma unroll
        for (int K = 0; K < D; ++K) rr2 += r[K] * r[K];
        if (rr2 == R(0)) continue;
        R rr = sqrt(rr2), w, dw;
        kern_wdw<R>(rr, inv_l, ad, w, dw);
        R gw[D], fac = -dw / rr, gt[D], rg = R(0);
#pragma unroll
        for (int K = 0; K < D; ++K) gw[K] = fac * r[K];
#pragma unroll
        for (int K = 0; K < D; ++K) {
            R s = R(0);
#pragma unroll
            for (int L2 = 0; L2 < D; ++L2) s += L[K * D + L2] * gw[L2];
            gt[K] = s;
            rg += r[K] * s;
        }
        R Vj = vol_at<R>(W, j);
        R F = rg / (rr2 * rr2), VF = Vj * F;
        R q[M], pv[M];
        qvec<D, R>(r, q);
#pragma unroll
        for (int a = 0; a < M; ++a) {
            R s = R(0);
#pragma unroll
            for (int K = 0; K < D; ++K) s += Ct[K * M + a] * r[K];
            pv[a] = q[a] - s;
        }
#pragma unroll
        for (int a = 0; a < M; ++a) {
            R vq = VF * q[a];
#pragma unroll
            for (int b = 0; b < M; ++b) Mm[a * M + b].add(vq * pv[b]);
#pragma unroll
            for (int K = 0; K < D; ++K) Q[a * D + K].add(vq * r[K]);
        }
        if (predictor) {
            // v_ij - r_ij . <grad v>_i cancels O(|grad v| r) down to O(|D v| r^2).
            // FP64 form: formed in FP64.  Mixed form: v_ij from the hi/lo velocities
            // (relative error ~u, as the FP64 difference rounded), r . <grad v> in
            // FP32; the remainder then carries ~5u |v_ij|, a relative error of
            // ~5u |v_ij| / |e| in e, which only enters the viscous term.
            if constexpr (MIXED) {
                float vij[D];
                if (tj == FLUID || P.slip) {
                    hilo_diff<D>(W.velhi[j], W.vello[j], vhi, vlo, vij);
                } else {
                    vij[0] = -(vhi.x + vlo.x);
                    if (D == 3) vij[1] = -(vhi.y + vlo.y);
                    vij[D - 1] = -(vhi.z + vlo.z);
                }
#pragma unroll
                for (int cc = 0; cc < D; ++cc) {
                    float rgv = 0.f;
#pragma unroll
                    for (int K = 0; K < D; ++K) rgv += r[K] * gvf[cc * D + K];
                    const R e = vij[cc] - rgv;
#pragma unroll
                    for (int a = 0; a < M; ++a) bv[a * D + cc].add(VF * q[a] * e);
                }
            } else {
                double vj[3] = {0.0, 0.0, 0.0};
                if (tj == FLUID || P.slip) load_vel<D>(c, j, vj);
#pragma unroll
                for (int cc = 0; cc < D; ++cc) {
                    double rgv = 0.0;
#pragma unroll
                    for (int K = 0; K < D; ++K) rgv += rd[K] * gvd[cc * D + K];
                    R e = (R)((vj[cc] - vi[cc]) - rgv);
#pragma unroll
                    for (int a = 0; a < M; ++a) bv[a * D + cc].add(VF * q[a] * e);
                }
            }
            // without the Smagorinsky model nu is nu_K everywhere and every
            // difference is zero (adding zeros leaves the compensated sums as they are)
            if (P.smag) {
                double nuj = tj == FLUID ? W.nu[j] : P.nu_k;
                R dn = (R)(nuj - nui);
#pragma unroll
                for (int K = 0; K < D; ++K) Gnu[K].add(Vj * dn * gw[K]);
            }
        }
    }
    double Md[M * M];
#pragma unroll
    for (int k = 0; k < M * M; ++k) Md[k] = (double)Mm[k].val();
    double ct[M];
    ctilde<D>(c.c3[i], c.sx[i], c.sy[i], ct);
    double acc[D] = {};
    int piv[M];
    if (predictor) {
        double Bv[M * D];
#pragma unroll
        for (int k = 0; k < M * D; ++k) Bv[k] = (double)bv[k].val();
        // M is factored once: D^v = 2 M^-1 b here, M^-T c~ for the pressure row below.
        // An isolated particle has no second derivatives; a free-surface particle
        // whose M_i cannot be factored (too few neighbours) loses its viscous
        // term; anywhere else a singular M_i is an error.
        const int fsi = W.fs[i];
        bool ok = fsi != 2 && lu_factor<M>(Md, piv);
        if (ok) lu_apply<M, D>(Md, piv, Bv);
        else {
            if (!fsi) set_error(W.status, VCT_ERR_SINGULAR, i);
#pragma unroll
            for (int k = 0; k < M * D; ++k) Bv[k] = 0.0;
        }
        // physical grad nu = J L sum V (nu_j - nu_i) grad w
        double gnh[D], gn[D];
#pragma unroll
        for (int K = 0; K < D; ++K) {
            double s = 0.0;
#pragma unroll
            for (int L2 = 0; L2 < D; ++L2) s += W.L[(int64_t)(K * D + L2) * cap + i] * (double)Gnu[L2].val();
            gnh[K] = s;
        }
        jac_apply<D>(c.J[i], c.sx[i], c.sy[i], gnh, gn);
        double G[D * D];  // G[I*D + cc] = d v_cc / d x_I
#pragma unroll
        for (int cc = 0; cc < D; ++cc) {
            double gh[D], g[D];
#pragma unroll
            for (int K = 0; K < D; ++K) gh[K] = W.gv[(int64_t)(cc * D + K) * cap + i];
            jac_apply<D>(c.J[i], c.sx[i], c.sy[i], gh, g);
#pragma unroll
            for (int I = 0; I < D; ++I) G[I * D + cc] = g[I];
        }
        const double c0i = c.c0[i];
#pragma unroll
        for (int cc = 0; cc < D; ++cc) {
            double lap = c0i * W.gv[(int64_t)(cc * D + (D - 1)) * cap + i];
#pragma unroll
            for (int a = 0; a < M; ++a) lap += ct[a] * 2.0 * Bv[a * D + cc];
            double term = 0.0;
#pragma unroll
            for (int J2 = 0; J2 < D; ++J2) term += (G[cc * D + J2] + G[J2 * D + cc]) * gn[J2];
            double g = cc == D - 1 ? -P.g : 0.0;
            acc[cc] = nui * lap + term + g;
            W.acc[(int64_t)cc * cap + i] = acc[cc];
            W.vstar[(int64_t)cc * cap + i] = vi[cc] + P.dt * acc[cc];
        }
        {
            double vs[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int cc = 0; cc < D; ++cc) vs[cc] = W.vstar[(int64_t)cc * cap + i];
            float4 lo;
            W.vshi[i] = f4_hilo_split(vs[0], D == 3 ? vs[1] : 0.0, vs[D - 1], lo);
            W.vslo[i] = lo;
        }
    }
    // pressure-equation row for unknowns (fluid, not free surface)
    if (!predictor || W.fs[i]) {
        if (predictor) W.pcnt[i] = -1;
        return;
    }
    double wv[M];
#pragma unroll
    for (int a = 0; a < M; ++a) wv[a] = ct[a];
    lu_apply_t<M>(Md, piv, wv);   // M^T w = c~ from the factors of M
    double u[D];
#pragma unroll
    for (int K = 0; K < D; ++K) {
        double s = 0.0;
#pragma unroll
        for (int a = 0; a < M; ++a) s += wv[a] * (double)Q[a * D + K].val();
        u[K] = s;
    }
    R wr[M], ur[D];
#pragma unroll
    for (int a = 0; a < M; ++a) wr[a] = (R)wv[a];
#pragma unroll
    for (int K = 0; K < D; ++K) ur[K] = (R)u[K];
    const R c0r = (R)c.c0[i];
    double diag = 0.0, wallrhs = 0.0, pw[D];
#pragma unroll
    for (int K = 0; K < D; ++K) pw[K] = 0.0;
    double pi_[3];
    load_phys<D>(c, i, pi_);
    int pc = 0;
    for (int k = 0; k < cnt; ++k) {
        int j = W.nbr[(int64_t)k * cap + i];
        int tj = c.type[j];
        if (tj == VIRTUAL) continue;
        R r[D], rr2 = R(0);
        pair_r<D, R>(c, W, j, xi, hfi, lfi, r);
#pragma unroll
        for (int K = 0; K < D; ++K) rr2 += r[K] * r[K];
        if (rr2 == R(0)) continue;
        R rr = sqrt(rr2), w, dw;
        kern_wdw<R>(rr, inv_l, ad, w, dw);
        R gw[D], fac = -dw / rr, gt[D], rg = R(0), ug = R(0);
#pragma unroll
        for (int K = 0; K < D; ++K) gw[K] = fac * r[K];
#pragma unroll
        for (int K = 0; K < D; ++K) {
            R s = R(0);
#pragma unroll
            for (int L2 = 0; L2 < D; ++L2) s += L[K * D + L2] * gw[L2];
            gt[K] = s;
            rg += r[K] * s;
            ug += ur[K] * s;
        }
        R F = rg / (rr2 * rr2), q[M], wq = R(0);
        qvec<D, R>(r, q);
#pragma unroll
        for (int a = 0; a < M; ++a) wq += wr[a] * q[a];
        R Vj = vol_at<R>(W, j);
        double aij = (double)(Vj * (c0r * gt[D - 1] + R(2) * F * wq - R(2) * ug));
        if (tj == FLUID) {
            diag -= aij;
            if (!W.fs[j]) {
                const int64_t q = ell_at<ell_group<D>()>(pc, i, cap);
                W.pcol[q] = j;
                if (P.precision == VCT_MIXED) W.pvalf[q] = (float)aij;
                else W.pval[q] = aij;
                ++pc;
            }
        } else {  // wall: p_ij = rho r_ij . f_i (Eq. PNC)
            double pj[3], s = 0.0;
            load_phys<D>(c, j, pj);
#pragma unroll
            for (int K = 0; K < D; ++K) {
                s += (pj[K] - pi_[K]) * acc[K];
                pw[K] += aij * P.rho * (pj[K] - pi_[K]);
            }
            wallrhs += aij * P.rho * s;
        }
    }
    W.pcnt[i] = pc;
    W.diag[i] = diag;
    W.wallrhs[i] = wallrhs;
#pragma unroll
    for (int K = 0; K < D; ++K) W.pwall[(int64_t)K * cap + i] = pw[K];
    atomicAdd((unsigned long long *)&W.counts[0], 1ull);
    atomicAdd((unsigned long long *)&W.counts[1], (unsigned long long)pc);
}

template <int D, typename R>
__global__ void __launch_bounds__(128, pass2_min_blocks<D>()) k_pass2(DevParams P, const Part c, Work W, int n,
                                               int predictor)
{
    pass2_body<D, R>(P, c, W, n, predictor, blockIdx.x);
}

// Pass 2 of the ISPH operator set (Table tab:case_names): the predictor with the
// 0th-order second derivatives of Eq. (sec_0th), D_a v = sum_j V_j k_a(r_ij) v_ij,
// and the pressure row c_trans . <D^ p>^(0): a_ij = V_j (c0 (L grad w)_z^ +
// sum_a c~_a k_a(r_ij)).  No moment matrix and no per-particle solve.
template <int D, typename R>
__device__ __forceinline__ void pass2_isph_body(const DevParams &P, const Part &c, const Work &W, int n, int bid_)
{
    if (step_failed(W.status)) return;
    constexpr int M = D == 2 ? 3 : 6;
    int i = bid_ * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (c.type[i] != FLUID) {
        W.pcnt[i] = -1;
        return;
    }
    const int64_t cap = W.cap;
    double xi[3], vi[3];
    load_hat<D>(c, i, xi);
    const float4 hfi = W.hatf[i], lfi = W.hatlo[i];
    load_vel<D>(c, i, vi);
    R L[D * D];
#pragma unroll
    for (int k = 0; k < D * D; ++k) L[k] = (R)W.L[(int64_t)k * cap + i];
    const double nui = W.nu[i];
    constexpr bool MIXED = sizeof(R) == sizeof(float);
    const float4 vhi = W.velhi[i], vlo = W.vello[i];
    Acc<R> Dv[M * D], Gnu[D];
    const R inv_l = (R)P.inv_l, ad = (R)P.ad;
    const int cnt = W.nbr_cnt[i];
    for (int k = 0; k < cnt; ++k) {
        int j = W.nbr[(int64_t)k * cap + i];
        int tj = c.type[j];
        if (tj == VIRTUAL) continue;
        R r[D], rr2 = R(0);
        pair_r<D, R>(c, W, j, xi, hfi, lfi, r);
#pragma unroll
        for (int K = 0; K < D; ++K) rr2 += r[K] * r[K];
        if (rr2 == R(0)) continue;
        R rr = sqrt(rr2), w, dw;
        kern_wdw<R>(rr, inv_l, ad, w, dw);
        const R fac = -dw / rr, Vj = vol_at<R>(W, j);
        R kw[M];
        er_weights<D, R>(r, rr2, fac, kw);
        R vij[D];
        if constexpr (MIXED) {
            float vf[D];
            if (tj == FLUID || P.slip) {
                hilo_diff<D>(W.velhi[j], W.vello[j], vhi, vlo, vf);
            } else {
                vf[0] = -(vhi.x + vlo.x);
                if (D == 3) vf[1] = -(vhi.y + vlo.y);
                vf[D - 1] = -(vhi.z + vlo.z);
            }
#pragma unroll
            for (int cc = 0; cc < D; ++cc) vij[cc] = vf[cc];
        } else {
            double vj[3] = {0.0, 0.0, 0.0};
            if (tj == FLUID || P.slip) load_vel<D>(c, j, vj);
#pragma unroll
            for (int cc = 0; cc < D; ++cc) vij[cc] = (R)(vj[cc] - vi[cc]);
        }
#pragma unroll
        for (int a = 0; a < M; ++a)
#pragma unroll
            for (int cc = 0; cc < D; ++cc) Dv[a * D + cc].add(Vj * kw[a] * vij[cc]);
        if (P.smag) {
            double nuj = tj == FLUID ? W.nu[j] : P.nu_k;
            R dn = (R)(nuj - nui);
#pragma unroll
            for (int K = 0; K < D; ++K) Gnu[K].add(Vj * dn * fac * r[K]);
        }
    }
    double ct[M];
    ctilde<D>(c.c3[i], c.sx[i], c.sy[i], ct);
    double acc[D];
    {
        double gnh[D], gn[D];
#pragma unroll
        for (int K = 0; K < D; ++K) {
            double s = 0.0;
#pragma unroll
            for (int L2 = 0; L2 < D; ++L2) s += W.L[(int64_t)(K * D + L2) * cap + i] * (double)Gnu[L2].val();
            gnh[K] = s;
        }
        jac_apply<D>(c.J[i], c.sx[i], c.sy[i], gnh, gn);
        double G[D * D];  // G[I*D + cc] = d v_cc / d x_I
#pragma unroll
        for (int cc = 0; cc < D; ++cc) {
            double gh[D], g[D];
#pragma unroll
            for (int K = 0; K < D; ++K) gh[K] = W.gv[(int64_t)(cc * D + K) * cap + i];
            jac_apply<D>(c.J[i], c.sx[i], c.sy[i], gh, g);
#pragma unroll
            for (int I = 0; I < D; ++I) G[I * D + cc] = g[I];
        }
        const double c0i = c.c0[i];
        const double dscale = W.fs[i] == 2 ? 0.0 : 1.0;   // isolated: no second derivatives
#pragma unroll
        for (int cc = 0; cc < D; ++cc) {
            double lap = c0i * W.gv[(int64_t)(cc * D + (D - 1)) * cap + i];
#pragma unroll
            for (int a = 0; a < M; ++a) lap += dscale * ct[a] * (double)Dv[a * D + cc].val();
            double term = 0.0;
#pragma unroll
            for (int J2 = 0; J2 < D; ++J2) term += (G[cc * D + J2] + G[J2 * D + cc]) * gn[J2];
            double g = cc == D - 1 ? -P.g : 0.0;
            acc[cc] = nui * lap + term + g;
            W.acc[(int64_t)cc * cap + i] = acc[cc];
            W.vstar[(int64_t)cc * cap + i] = vi[cc] + P.dt * acc[cc];
        }
        double vs[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int cc = 0; cc < D; ++cc) vs[cc] = W.vstar[(int64_t)cc * cap + i];
        float4 lo;
        W.vshi[i] = f4_hilo_split(vs[0], D == 3 ? vs[1] : 0.0, vs[D - 1], lo);
        W.vslo[i] = lo;
    }
    if (W.fs[i]) {
        W.pcnt[i] = -1;
        return;
    }
    R ctr[M];
#pragma unroll
    for (int a = 0; a < M; ++a) ctr[a] = (R)ct[a];
    const R c0r = (R)c.c0[i];
    double diag = 0.0, wallrhs = 0.0, pw[D];
#pragma unroll
    for (int K = 0; K < D; ++K) pw[K] = 0.0;
    double pi_[3];
    load_phys<D>(c, i, pi_);
    int pc = 0;
    for (int k = 0; k < cnt; ++k) {
        int j = W.nbr[(int64_t)k * cap + i];
        int tj = c.type[j];
        if (tj == VIRTUAL) continue;
        R r[D], rr2 = R(0);
        pair_r<D, R>(c, W, j, xi, hfi, lfi, r);
#pragma unroll
        for (int K = 0; K < D; ++K) rr2 += r[K] * r[K];
        if (rr2 == R(0)) continue;
        R rr = sqrt(rr2), w, dw;
        kern_wdw<R>(rr, inv_l, ad, w, dw);
        const R fac = -dw / rr;
        R kw[M], gz = R(0), sk = R(0);
        er_weights<D, R>(r, rr2, fac, kw);
#pragma unroll
        for (int L2 = 0; L2 < D; ++L2) gz += L[(D - 1) * D + L2] * fac * r[L2];
#pragma unroll
        for (int a = 0; a < M; ++a) sk += ctr[a] * kw[a];
        double aij = (double)(vol_at<R>(W, j) * (c0r * gz + sk));
        if (tj == FLUID) {
            diag -= aij;
            if (!W.fs[j]) {
                const int64_t q = ell_at<ell_group<D>()>(pc, i, cap);
                W.pcol[q] = j;
                if (P.precision == VCT_MIXED) W.pvalf[q] = (float)aij;
                else W.pval[q] = aij;
                ++pc;
            }
        } else {  // wall: p_ij = rho r_ij . f_i (Eq. PNC)
            double pj[3], s2 = 0.0;
            load_phys<D>(c, j, pj);
#pragma unroll
            for (int K = 0; K < D; ++K) {
                s2 += (pj[K] - pi_[K]) * acc[K];
                pw[K] += aij * P.rho * (pj[K] - pi_[K]);
            }
            wallrhs += aij * P.rho * s2;
        }
    }
    W.pcnt[i] = pc;
    W.diag[i] = diag;
    W.wallrhs[i] = wallrhs;
#pragma unroll
    for (int K = 0; K < D; ++K) W.pwall[(int64_t)K * cap + i] = pw[K];
    atomicAdd((unsigned long long *)&W.counts[0], 1ull);
    atomicAdd((unsigned long long *)&W.counts[1], (unsigned long long)pc);
}

template <int D, typename R>
__global__ void __launch_bounds__(128) k_pass2_isph(DevParams P, const Part c, Work W, int n)
{
    pass2_isph_body<D, R>(P, c, W, n, blockIdx.x);
}

void launch_pass2(const DevParams &P, Part cur, Work W, int64_t n, int predictor,
                  cudaStream_t st)
{
    unsigned g = (unsigned)((n + 127) / 128);
    if (P.operators == 1 && predictor) {
        if (P.dim == 2) {
            if (P.precision == VCT_MIXED) k_pass2_isph<2, float><<<g, 128, 0, st>>>(P, cur, W, (int)n);
            else k_pass2_isph<2, double><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        } else {
            if (P.precision == VCT_MIXED) k_pass2_isph<3, float><<<g, 128, 0, st>>>(P, cur, W, (int)n);
            else k_pass2_isph<3, double><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        }
        return;
    }
    if (P.dim == 2) {
        if (P.precision == VCT_MIXED) k_pass2<2, float><<<g, 128, 0, st>>>(P, cur, W, (int)n, predictor);
        else k_pass2<2, double><<<g, 128, 0, st>>>(P, cur, W, (int)n, predictor);
    } else {
        if (P.precision == VCT_MIXED) k_pass2<3, float><<<g, 128, 0, st>>>(P, cur, W, (int)n, predictor);
        else k_pass2<3, double><<<g, 128, 0, st>>>(P, cur, W, (int)n, predictor);
    }
}

// ---------------------------------------------------------------------------
// a7 (right side): b_i = rho/dt tr(J <grad^ (x) v*>) + gamma (rho Jbar/J - rho^)/dt^2
//                       - (wall terms of Eq. PNC)
// A wall neighbour carries v_wall + dt f_i, the intermediate velocity implied by
// the acceleration Eq. (PNC) assumes.
// ---------------------------------------------------------------------------
template <int D, typename R>
__device__ __forceinline__ void rhs_body(const DevParams &P, const Part &c, const Work &W, int n, int bid_)
{
    if (step_failed(W.status)) return;
    int i = bid_ * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t cap = W.cap;
    if (c.type[i] != FLUID || W.fs[i]) {
        W.bvec[i] = 0.0;
        W.kx[i] = 0.0;
        return;
    }
    double xi[3], vsi[D], acci[D];
    load_hat<D>(c, i, xi);
    const float4 hfi = W.hatf[i], lfi = W.hatlo[i];
#pragma unroll
    for (int cc = 0; cc < D; ++cc) {
        vsi[cc] = W.vstar[(int64_t)cc * cap + i];
        acci[cc] = W.acc[(int64_t)cc * cap + i];
    }
    R wall_dv[D];   // a wall neighbour's v_j - v*_i, the same for every wall neighbour
#pragma unroll
    for (int cc = 0; cc < D; ++cc) wall_dv[cc] = (R)(P.dt * acci[cc] - vsi[cc]);
    const float4 vshi_i = W.vshi[i], vslo_i = W.vslo[i];
    Acc<R> X[D * D];
    const R inv_l = (R)P.inv_l, ad = (R)P.ad;
    const int cnt = W.nbr_cnt[i];
    for (int k = 0; k < cnt; ++k) {
        int j = W.nbr[(int64_t)k * cap + i];
        int tj = c.type[j];
        if (tj == VIRTUAL) continue;
        R r[D], rr2 = R(0);
        pair_r<D, R>(c, W, j, xi, hfi, lfi, r);
#pragma unroll
        for (int K = 0; K < D; ++K) rr2 += r[K] * r[K];
        if (rr2 == R(0)) continue;
        R rr = sqrt(rr2), w, dw;
        kern_wdw<R>(rr, inv_l, ad, w, dw);
        R fac = -dw / rr, Vj = vol_at<R>(W, j);
        R dv[D];
        if (tj != FLUID) {
#pragma unroll
            for (int cc = 0; cc < D; ++cc) dv[cc] = wall_dv[cc];
            if (P.slip) {   // a free-slip wall carries its velocity + dt f_i
                double vj[3] = {0.0, 0.0, 0.0};
                load_vel<D>(c, j, vj);
#pragma unroll
                for (int cc = 0; cc < D; ++cc) dv[cc] += (R)vj[cc];
            }
        } else if constexpr (sizeof(R) == sizeof(float)) {   // mixed: hi/lo differences
            hilo_diff<D>(W.vshi[j], W.vslo[j], vshi_i, vslo_i, dv);
        } else {
#pragma unroll
            for (int cc = 0; cc < D; ++cc) dv[cc] = (R)(W.vstar[(int64_t)cc * cap + j] - vsi[cc]);
        }
#pragma unroll
        for (int cc = 0; cc < D; ++cc) {
            R e = Vj * dv[cc] * fac;
#pragma unroll
            for (int K = 0; K < D; ++K) X[cc * D + K].add(e * r[K]);
        }
    }
    double div = 0.0;
#pragma unroll
    for (int cc = 0; cc < D; ++cc) {
        double gh[D], g[D];
#pragma unroll
        for (int K = 0; K < D; ++K) {
            double s = 0.0;
#pragma unroll
            for (int L2 = 0; L2 < D; ++L2) s += W.L[(int64_t)(K * D + L2) * cap + i] * (double)X[cc * D + L2].val();
            gh[K] = s;
        }
        jac_apply<D>(c.J[i], c.sx[i], c.sy[i], gh, g);
        div += g[cc];
    }
    double fac = P.volume_mode == 0 ? 1.0 : c.jbar[i] / c.J[i];
    double rhs = P.rho / P.dt * div + P.gamma * (P.rho * fac - W.rho_hat[i]) / (P.dt * P.dt);
    W.bvec[i] = rhs - W.wallrhs[i];
    // initial guess: p^N, or its extrapolation from the previous steps when this
    // particle's pressure is exactly what this context's previous step left (the
    // caller continued it): 2 p^N - p^(N-1), or 3 p^N - 3 p^(N-1) + p^(N-2)
    const int o = c.orig[i];
    const double pn = c.p[i];
    double x0 = pn;
    if (pn == W.p_last[o]) {
        const double p1 = W.p_prev[o], p2 = W.p_prev2[o];
        x0 = (P.pguess >= 2 && isfinite(p2)) ? 3.0 * pn - 3.0 * p1 + p2 : 2.0 * pn - p1;
    }
    if (P.pguess == 0) x0 = pn;
    W.kx[i] = x0;
}

template <int D, typename R>
__global__ void __launch_bounds__(128) k_rhs(DevParams P, const Part c, Work W, int n)
{
    rhs_body<D, R>(P, c, W, n, blockIdx.x);
}

void launch_rhs(const DevParams &P, Part cur, Work W, int64_t n, cudaStream_t st)
{
    unsigned g = (unsigned)((n + 127) / 128);
    if (P.dim == 2) {
        if (P.precision == VCT_MIXED) k_rhs<2, float><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        else k_rhs<2, double><<<g, 128, 0, st>>>(P, cur, W, (int)n);
    } else {
        if (P.precision == VCT_MIXED) k_rhs<3, float><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        else k_rhs<3, double><<<g, 128, 0, st>>>(P, cur, W, (int)n);
    }
}

// ---------------------------------------------------------------------------
// a8: pressure solve.  FP64 iterative refinement on the true residual
// f = b - A x around an inner BiCGSTAB (van der Vorst 1992) in precision T:
// T = double for the FP64 form (one pass to krylov_rtol), T = float with
// FP32-stored coefficients for the mixed form (each pass to 1e-4, then a new
// FP64 residual).  Everything runs in one cooperative persistent launch.
// Two grid barriers per inner iteration: the recurrences are rearranged so that
// (rh, r_new) = (rh, s) - w (rh, t) and |r_new|^2 = (s,s) - 2w (t,s) + w^2 (t,t)
// come out of the second reduction, the x/r update of iteration k is applied at
// the start of iteration k+1, and the new search direction and s are formed on
// the fly inside the two operator products.  Dot products: per-block partials
// summed in the same order by every block (identical scalars everywhere,
// bit-reproducible runs).
// ---------------------------------------------------------------------------
constexpr int KT = 256;
// Solver blocks per SM the large-system and the batched solvers are compiled
// for (register budget 65536 / (KT x this)).  Measured, krylov ms per step:
// 2.1M-particle 3-D beach, V(0,1) cycles, 2 blocks 121.6, 3 blocks 114.1, 4
// blocks 116.2 (after the later changes: 3 blocks 85.1, 4 blocks 95.8); 64 2-D
// scenarios side by side, 2 blocks 29.4, 3 blocks 18.8 (later: 3 blocks 100.7,
// 4 blocks 105.4 M particle-updates/s for the whole step).
#ifndef VCT_KMG_MINB
#define VCT_KMG_MINB 3
#endif
#ifndef VCT_KBATCH_MINB
#define VCT_KBATCH_MINB 4   // the batch in the large-system form (the small-system form: 2)
#endif

__device__ __forceinline__ unsigned ld_acquire(const unsigned int *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned atom_add_release(unsigned int *p, unsigned v)
{
    unsigned o;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(o) : "l"(p), "r"(v) : "memory");
    return o;
}

// Grid barrier for a cooperative launch (all blocks resident), one atomic per
// block: block 0 adds 2^31 - (nblocks - 1), every other block adds 1, so the
// word's top bit flips exactly when the last block arrives; each block waits
// for the top bit to differ from the value it saw.  The word needs no reset.
// Spins are bounded: on timeout the block records status[2], and every block
// leaves at its next barrier, so the kernel always ends.
// vb: the block's index among the nblocks that share the barrier word (the
// grid, or a batched solve's subset of it); limit: polls before a wait gives
// up (the context's spin limit, by default ~1-2 s).
__device__ bool grid_barrier(unsigned int *bar, unsigned nblocks, int32_t *status, unsigned vb,
                             unsigned long long limit)
{
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned inc = vb == 0 ? 0x80000000u - (nblocks - 1u) : 1u;
        unsigned old = atom_add_release(bar, inc);
        unsigned long long spins = 0;
        while (((ld_acquire(bar) ^ old) & 0x80000000u) == 0u) {
            if (++spins > limit) {
                ok = 0;
                atomicExch(status + 2, 1);
                // also the call's error code: the steps queued after this one become
                // no-ops and the caller's state is not written back
                set_error(status, VCT_ERR_TIMEOUT, -1);
                break;
            }
        }
        if (*(volatile int32_t *)(status + 2)) ok = 0;
        ok_sh = ok;
    }
    __syncthreads();
    return ok_sh != 0;
}


// Per-block partial sums, stored k-major: partial[k * PSTRIDE + block].
constexpr int PSTRIDE = 4096;

template <int NV>
__device__ void block_partials(const double (&v)[NV], double *partial, unsigned vb)
{
    __shared__ double sh[NV][KT / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sh[k][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < KT / 32; ++w) s += sh[threadIdx.x][w];
        partial[(int64_t)threadIdx.x * PSTRIDE + vb] = s;
    }
}

template <int NV>
__device__ __forceinline__ void block_partials(const double (&v)[NV], double *partial)
{
    block_partials<NV>(v, partial, blockIdx.x);
}

// Sum the per-block partials: every thread of the block loads a strided
// subset (independent, coalesced loads), then a fixed-order tree.  The order
// does not depend on the block, so every block gets the same bits.
template <int NV>
__device__ void grid_totals(const double *partial, unsigned nblocks, double (&out)[NV])
{
    __shared__ double red[NV][KT / 32];
    __shared__ double tot[NV];
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
    for (unsigned b = threadIdx.x; b < nblocks; b += KT)
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] += __ldcg(partial + (int64_t)k * PSTRIDE + b);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double x = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[k][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < KT / 32; ++w) s += red[threadIdx.x][w];
        tot[threadIdx.x] = s;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = tot[k];
    __syncthreads();
}

template <typename CT>
__device__ __forceinline__ CT coef(const Work &W, int64_t k);
template <>
__device__ __forceinline__ double coef<double>(const Work &W, int64_t k) { return W.pval[k]; }
template <>
__device__ __forceinline__ float coef<float>(const Work &W, int64_t k) { return W.pvalf[k]; }

// Sum over the G lanes of a row group (G consecutive lanes of a warp).  The
// shuffle names only the group's lanes: the groups of one warp work on
// different rows and may leave the row loop at different times, while the
// lanes of one group always share the row, its coefficient count and the trip
// count, so they reach every shuffle together.
template <int G, typename T>
__device__ __forceinline__ T group_sum(T v)
{
    static_assert(G >= 2 && G <= 32 && (G & (G - 1)) == 0, "G: power of two <= 32");
    const unsigned lane = threadIdx.x & 31u;
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(unsigned)(G - 1)));
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(gmask, v, o, G);
    return v;
}

// Dot of row i with a gathered vector: lane lg of the row's group takes slots
// lg, lg+G, ...  The first NS slots' columns and coefficients are loaded before
// the row's count is known (ELL slots below max_nbr are always allocated), so a
// row costs one round trip for its operator and one for the gathers.
template <typename T, typename CT, int G, int NS, typename GetX>
__device__ __forceinline__ T row_dot(const Work &W, int i, int pc, int lg, GetX getx)
{
    const int64_t cap = W.cap;
    int jj[NS];
    CT aa[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int kk = lg + s * G;
        jj[s] = 0;
        aa[s] = CT(0);
        if (kk < W.max_nbr) {
            const int64_t q = ell_at<G>(kk, i, cap);
            jj[s] = W.pcol[q];
            aa[s] = coef<CT>(W, q);
        }
    }
    T acc = T(0);
#pragma unroll
    for (int s = 0; s < NS; ++s)
        if (lg + s * G < pc) acc += (T)aa[s] * getx(jj[s]);
    for (int kk = lg + NS * G; kk < pc; kk += G) {
        const int64_t q = ell_at<G>(kk, i, cap);
        acc += (T)coef<CT>(W, q) * getx(W.pcol[q]);
    }
    return acc;
}

// As row_dot, with the row's count loaded in the same round trip as its operator.
template <typename T, typename CT, int G, int NS, typename GetX>
__device__ __forceinline__ T row_dot_pc(const Work &W, int i, int lg, int &pc_out, GetX getx)
{
    const int64_t cap = W.cap;
    const int pc = W.pcnt[i];
    int jj[NS];
    CT aa[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int kk = lg + s * G;
        jj[s] = 0;
        aa[s] = CT(0);
        if (kk < W.max_nbr) {
            const int64_t q = ell_at<G>(kk, i, cap);
            jj[s] = W.pcol[q];
            aa[s] = coef<CT>(W, q);
        }
    }
    T acc = T(0);
#pragma unroll
    for (int s = 0; s < NS; ++s)
        if (lg + s * G < pc) acc += (T)aa[s] * getx(jj[s]);
    for (int kk = lg + NS * G; kk < pc; kk += G) {
        const int64_t q = ell_at<G>(kk, i, cap);
        acc += (T)coef<CT>(W, q) * getx(W.pcol[q]);
    }
    pc_out = pc;
    return acc;
}

// G lanes per row; the row's scalar work is repeated by every lane of the group
// (same addresses, broadcast loads) and only lane 0 writes.  Dot-product
// partials are accumulated per thread in T and summed per block in FP64.
template <typename T, typename CT, int G, int NS>
__global__ void __launch_bounds__(KT) k_krylov(Work W, int n, int maxit, double rtol,
                                               double inner_floor, int32_t *iters_out,
                                               double *resid_out)
{
    if (step_failed(W.status)) return;
    const unsigned nb = gridDim.x;
    const int lg = threadIdx.x & (G - 1);
    const bool lead = lg == 0;
    const int ngroups = (gridDim.x * blockDim.x) / G;
    const int g0 = (blockIdx.x * blockDim.x + threadIdx.x) / G;
    double *x = W.kx, *f = W.kf;
    T *r = (T *)W.kr, *rh = (T *)W.krh, *s = (T *)W.ks, *t = (T *)W.kt, *dl = (T *)W.kd;
    T *pold = (T *)W.kp0, *pnew = (T *)W.kp1, *vold = (T *)W.kv0, *vnew = (T *)W.kv1;
    int total_it = 0;
    bool fail = false;
    double bn = 0.0, rn = 0.0;
    for (int outer = 0;; ++outer) {
        // true residual in FP64: f = b - A x
        double part[2] = {0.0, 0.0};
        for (int i = g0; i < n; i += ngroups) {
            const int pc = W.pcnt[i];
            if (pc < 0) continue;
            double ax = row_dot<double, CT, G, NS>(W, i, pc, lg, [&](int j) { return __ldcg(x + j); });
            ax = group_sum<G>(ax);
            if (lead) {
                double bi = W.bvec[i], fi = bi - (ax + W.diag[i] * x[i]);
                f[i] = fi;
                part[0] += fi * fi;
                part[1] += bi * bi;
            }
        }
        block_partials<2>(part, W.partial);
        if (!grid_barrier(W.bar, nb, W.status, blockIdx.x, W.spin_limit)) return;
        double tot[2];
        grid_totals<2>(W.partial, nb, tot);
        rn = sqrt(tot[0]);
        bn = sqrt(tot[1]);
        if (bn == 0.0) {
            for (int i = g0; i < n; i += ngroups)
                if (lead) x[i] = 0.0;
            rn = 0.0;
            break;
        }
        if (rn <= rtol * bn) break;
        if (total_it >= maxit || outer >= 64) {
            fail = true;
            break;
        }
        // inner solve A d = f in precision T, to |r| <= tol_in |f|
        const double fn = rn, tol_in = fmax(rtol * bn / rn, inner_floor);
        double rho = fn * fn, rho_old = 1.0, alpha = 1.0, omega = 1.0;
        double pend_a = 0.0, pend_w = 0.0;   // update of the last completed iteration
        bool first = true, have_pend = false;
        for (;;) {
            if (total_it >= maxit) break;
            ++total_it;
            const double beta = first ? 0.0 : (rho / rho_old) * (alpha / omega);
            const T tb = (T)beta, tw = (T)omega, ta = (T)alpha;
            // phase A: apply the pending update, p_new = r + beta (p - w v), v_new = A p_new
            T pa = T(0);
            for (int i = g0; i < n; i += ngroups) {
                const int pc = W.pcnt[i];
                if (pc < 0) continue;
                T acc;
                if (first)
                    acc = row_dot<T, CT, G, NS>(W, i, pc, lg, [&](int j) { return (T)__ldcg(f + j); });
                else
                    acc = row_dot<T, CT, G, NS>(W, i, pc, lg, [&](int j) {
                        return (__ldcg(s + j) - tw * __ldcg(t + j)) +
                               tb * (__ldcg(pold + j) - tw * __ldcg(vold + j));
                    });
                acc = group_sum<G>(acc);
                if (lead) {
                    T ri, pn;
                    if (first) {
                        ri = (T)f[i];
                        pn = ri;
                        rh[i] = ri;
                        dl[i] = T(0);
                    } else {
                        const T si = s[i], po = pold[i];
                        ri = si - tw * t[i];
                        pn = ri + tb * (po - tw * vold[i]);
                        dl[i] += ta * po + tw * si;
                    }
                    acc += (T)W.diag[i] * pn;
                    r[i] = ri;
                    pnew[i] = pn;
                    vnew[i] = acc;
                    pa += rh[i] * acc;
                }
            }
            {
                double pd[1] = {(double)pa};
                block_partials<1>(pd, W.partial);
            }
            if (!grid_barrier(W.bar, nb, W.status, blockIdx.x, W.spin_limit)) return;
            double tv[1];
            grid_totals<1>(W.partial, nb, tv);
            first = false;
            have_pend = false;
            if (tv[0] == 0.0) {
                fail = true;
                break;
            }
            alpha = rho / tv[0];
            const T ta2 = (T)alpha;
            // phase B: s = r - alpha v_new, t = A s; partials (t,s) (t,t) (s,s) (rh,s) (rh,t)
            T pb0 = T(0), pb1 = T(0), pb2 = T(0), pb3 = T(0), pb4 = T(0);
            for (int i = g0; i < n; i += ngroups) {
                const int pc = W.pcnt[i];
                if (pc < 0) continue;
                T acc = row_dot<T, CT, G, NS>(W, i, pc, lg, [&](int j) {
                    return __ldcg(r + j) - ta2 * __ldcg(vnew + j);
                });
                acc = group_sum<G>(acc);
                if (lead) {
                    const T si = r[i] - ta2 * vnew[i], hi = rh[i];
                    acc += (T)W.diag[i] * si;
                    s[i] = si;
                    t[i] = acc;
                    pb0 += acc * si;
                    pb1 += acc * acc;
                    pb2 += si * si;
                    pb3 += hi * si;
                    pb4 += hi * acc;
                }
            }
            {
                double pd[5] = {(double)pb0, (double)pb1, (double)pb2, (double)pb3, (double)pb4};
                block_partials<5>(pd, W.partial);
            }
            if (!grid_barrier(W.bar, nb, W.status, blockIdx.x, W.spin_limit)) return;
            double tq[5];
            grid_totals<5>(W.partial, nb, tq);
            T *tp = pold; pold = pnew; pnew = tp;
            tp = vold; vold = vnew; vnew = tp;
            have_pend = true;
            pend_a = alpha;
            if (sqrt(tq[2]) <= tol_in * fn) {   // s already small: x += alpha p
                pend_w = 0.0;
                break;
            }
            if (tq[1] == 0.0) {
                pend_w = 0.0;
                fail = true;
                break;
            }
            omega = tq[0] / tq[1];
            pend_w = omega;
            rho_old = rho;
            rho = tq[3] - omega * tq[4];
            double rr = tq[2] - 2.0 * omega * tq[0] + omega * omega * tq[1];
            if (sqrt(fmax(rr, 0.0)) <= tol_in * fn || rho == 0.0) break;
        }
        // apply the last update and x += d (FP64)
        const T fa = (T)pend_a, fw = (T)pend_w;
        for (int i = g0; i < n; i += ngroups) {
            if (!lead || W.pcnt[i] < 0) continue;
            T d = dl[i];
            if (have_pend) d += fa * pold[i] + fw * s[i];
            x[i] += (double)d;
        }
        if (!grid_barrier(W.bar, nb, W.status, blockIdx.x, W.spin_limit)) return;
        if (fail) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (fail) set_error(W.status, VCT_ERR_NOCONV, -1);
        iters_out[0] += total_it;
        if (total_it > iters_out[1]) iters_out[1] = total_it;
        iters_out[2] = total_it;
        *resid_out = bn > 0.0 ? rn / bn : 0.0;
    }
}

// 2-D: 4 lanes per row (~20 coefficients, 5 slots each); 3-D: 8 lanes (~56, 7 slots).
static const void *krylov_fn(int precision, int dim)
{
    if (precision == VCT_MIXED)
        return dim == 2 ? (const void *)k_krylov<float, float, 4, 5>
                        : (const void *)k_krylov<float, float, 8, 7>;
    return dim == 2 ? (const void *)k_krylov<double, double, 4, 5>
                    : (const void *)k_krylov<double, double, 8, 7>;
}

int krylov_coop_blocks(int precision, int dim)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, krylov_fn(precision, dim), KT, 0);
    if (per > 4) per = 4;
    int nb = sms * per;
    return nb < PSTRIDE ? nb : PSTRIDE;
}

int launch_krylov(const DevParams &P, Part cur, Work W, int64_t n, int step_slot,
                  int nblocks_coop, cudaStream_t st)
{
    (void)cur;
    (void)step_slot;
    int nn = (int)n, maxit = P.max_iter;
    double rtol = P.rtol, floor_ = P.inner_floor;
    int32_t *it_out = W.kiters;
    double *res_out = W.kresid;
    // a grid no larger than the rows need: fewer arrivals per barrier
    const int G = P.dim == 2 ? 4 : 8;
    int64_t want = (n * G + KT - 1) / KT;
    int nblk = (int)(want < nblocks_coop ? want : nblocks_coop);
    if (nblk < 1) nblk = 1;
    void *args[] = {(void *)&W, (void *)&nn, (void *)&maxit, (void *)&rtol, (void *)&floor_,
                    (void *)&it_out, (void *)&res_out};
    cudaMemsetAsync(W.bar, 0, 2 * sizeof(unsigned int), st);   // fresh barrier word
    cudaError_t e = cudaLaunchCooperativeKernel(krylov_fn(P.precision, P.dim), dim3(nblk),
                                                dim3(KT), args, 0, st);
    return e == cudaSuccess ? 0 : (int)e;
}

// ---------------------------------------------------------------------------
// a8 preconditioner: aggregation multigrid on the cell grid.
// Level 1 nodes are the neighbour-search cells (their particles are contiguous
// after the sort); the prolongation is piecewise constant, so the Galerkin
// operator of level 1 sums the pressure-equation coefficients between cells,
// giving a 3^d-point stencil; level l+1 aggregates 2 x 2 (x 2) nodes of level
// l the same way.  The V(1,1) cycle uses damped Jacobi; every neighbour value a
// phase needs is formed on the fly, so each level costs one grid barrier going
// down and one coming up.  Levels with at most 2048 nodes run inside block 0.
// All sums run in a fixed order (no floating-point atomics).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mg_coords(const MG &M, int l, int I, int &cx, int &cy, int &cz)
{
    const int nx = M.dims[l][0], ny = M.dims[l][1];
    cx = I % nx;
    int tq = I / nx;
    cy = tq % ny;
    cz = tq / ny;
}

template <int D>
__device__ __forceinline__ int stencil_index(int dx, int dy, int dz)
{
    return D == 2 ? (dz + 1) * 3 + (dx + 1) : ((dz + 1) * 3 + (dy + 1)) * 3 + (dx + 1);
}

// Add v to the stencil entry o, keeping the S accumulators in registers (a
// dynamically indexed array would live in local memory).
template <int S>
__device__ __forceinline__ void stencil_add(float (&acc)[S], int o, float v)
{
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] += s == o ? v : 0.f;
}

// One warp per cell: the lanes take the slots of the cell's rows in turn and
// the 3^d sums are reduced across the warp in a fixed order.
template <int D>
__device__ __forceinline__ void mg_level1_body(const Work &W, const MG &M, int mixed, int bid_)
{
    if (step_failed(W.status)) return;
    constexpr int S = D == 2 ? 9 : 27;
    const int N = M.n[1];
    const int lane = threadIdx.x & 31;
    const int I = (int)((bid_ * (unsigned)blockDim.x + threadIdx.x) >> 5);
    if (I >= N) return;
    float acc[S];
#pragma unroll
    for (int o = 0; o < S; ++o) acc[o] = 0.f;
    int cx, cy, cz;
    mg_coords(M, 1, I, cx, cy, cz);
    const int a = W.cell_start[I], b = W.cell_start[I + 1];
    const int64_t cap = W.cap;
    int rows = 0;
    double center = 0.0;
    for (int i = a; i < b; ++i) {
        const int pc = W.pcnt[i];
        if (pc < 0) continue;
        ++rows;
        center += W.diag[i];
        for (int k = lane; k < pc; k += 32) {
            const int64_t q = ell_at<ell_group<D>()>(k, i, cap);
            const int j = W.pcol[q];
            const float av = mixed ? W.pvalf[q] : (float)W.pval[q];
            int jx, jy, jz;
            mg_coords(M, 1, W.cellid[j], jx, jy, jz);
            stencil_add<S>(acc, stencil_index<D>(jx - cx, jy - cy, jz - cz), av);
        }
    }
#pragma unroll
    for (int o = 0; o < S; ++o)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc[o] += __shfl_xor_sync(0xffffffffu, acc[o], off);
    if (lane != 0) return;
    const int cidx = stencil_index<D>(0, 0, 0);
    acc[cidx] += (float)center;
    float *A = M.offA[1] + W.mg_pool;
    float *v = M.offv[1] + W.mg_pool;
#pragma unroll
    for (int o = 0; o < S; ++o) A[(int64_t)o * N + I] = acc[o];
    v[I] = (rows > 0 && acc[cidx] != 0.f) ? 1.f / acc[cidx] : 0.f;   // dinv
}

template <int D>
__global__ void k_mg_level1(Work W, MG M, int mixed)
{
    mg_level1_body<D>(W, M, mixed, blockIdx.x);
}

// Row-cell operator of the large-system form's V(0,1) cycle: for every unknown
// row i and each of the 3^d cells around its own, the sum of the row's
// coefficients on the particles of that cell (the diagonal in its own cell's
// entry), B[o][i] = sum over k in cell(i) + o of a_ik.  For a correction
// prolonged from the cells, zb_k = zu(cell(k)), (A zb)_i = sum_o B[o][i]
// zu(cell(i) + o): the fine post-smoothing then reads 3^d values per row
// instead of the row's coefficients and one gather per neighbour.  The lanes
// of a row's group take its slots in turn; the 3^d sums are reduced across the
// group in a fixed order.
template <int D>
__device__ __forceinline__ void mg_rowcell_body(const Work &W, const MG &M, int n, int mixed, int bid_)
{
    if (step_failed(W.status)) return;
    constexpr int S = D == 2 ? 9 : 27, G = ell_group<D>();
    const int lg = threadIdx.x & (G - 1);
    const int i = (int)((bid_ * (unsigned)blockDim.x + threadIdx.x) / G);
    if (i >= n) return;
    const int pc = W.pcnt[i];   // the same for the row's whole group
    if (pc < 0) return;
    float acc[S];
#pragma unroll
    for (int o = 0; o < S; ++o) acc[o] = 0.f;
    int cx, cy, cz;
    mg_coords(M, 1, W.cellid[i], cx, cy, cz);
    const int64_t cap = W.cap;
    for (int kk = lg; kk < pc; kk += G) {
        const int64_t q = ell_at<G>(kk, i, cap);
        const int j = W.pcol[q];
        const float av = mixed ? W.pvalf[q] : (float)W.pval[q];
        int jx, jy, jz;
        mg_coords(M, 1, W.cellid[j], jx, jy, jz);
        stencil_add<S>(acc, stencil_index<D>(jx - cx, jy - cy, jz - cz), av);
    }
#pragma unroll
    for (int o = 0; o < S; ++o) acc[o] = group_sum<G>(acc[o]);
    if (lg != 0) return;
    acc[stencil_index<D>(0, 0, 0)] += (float)W.diag[i];
#pragma unroll
    for (int o = 0; o < S; ++o) W.mg_B[(int64_t)o * cap + i] = acc[o];
}

template <int D>
__global__ void k_mg_rowcell(Work W, MG M, int n, int mixed)
{
    mg_rowcell_body<D>(W, M, n, mixed, blockIdx.x);
}

// Level 1 from the row-cell operator: the cell's stencil entry o is the sum of
// B[o][i] over its unknown rows, the Galerkin sum the warp-per-cell form
// gathers from the coefficients (B's own-cell entry holds the diagonal).  One
// thread per cell, the cell's rows in order.
template <int D>
__device__ __forceinline__ void mg_level1_rc_body(const Work &W, const MG &M, int bid_)
{
    if (step_failed(W.status)) return;
    constexpr int S = D == 2 ? 9 : 27;
    const int N = M.n[1];
    const int I = bid_ * blockDim.x + threadIdx.x;
    if (I >= N) return;
    const int a = W.cell_start[I], b = W.cell_start[I + 1];
    const int64_t cap = W.cap;
    float acc[S];
#pragma unroll
    for (int o = 0; o < S; ++o) acc[o] = 0.f;
    int rows = 0;
    for (int i = a; i < b; ++i) {
        if (W.pcnt[i] < 0) continue;
        ++rows;
#pragma unroll
        for (int o = 0; o < S; ++o) acc[o] += W.mg_B[(int64_t)o * cap + i];
    }
    float *A = W.mg_pool + M.offA[1];
#pragma unroll
    for (int o = 0; o < S; ++o) A[(int64_t)o * N + I] = acc[o];
    const float cc = acc[stencil_index<D>(0, 0, 0)];
    W.mg_pool[M.offv[1] + I] = (rows > 0 && cc != 0.f) ? 1.f / cc : 0.f;   // dinv
}

template <int D>
__global__ void k_mg_level1_rc(Work W, MG M)
{
    mg_level1_rc_body<D>(W, M, blockIdx.x);
}

// Node Ic of level l+1 from level l: sums of the children's stencils.
template <int D>
__device__ void coarsen_node(const Work &W, const MG &M, int l, int Ic)
{
    constexpr int S = D == 2 ? 9 : 27;
    const int Nc = M.n[l + 1], Nf = M.n[l];
    float acc[S];
#pragma unroll
    for (int o = 0; o < S; ++o) acc[o] = 0.f;
    int px, py, pz;
    mg_coords(M, l + 1, Ic, px, py, pz);
    const float *Af = W.mg_pool + M.offA[l];
    const float *vf = W.mg_pool + M.offv[l];
    const int fx = M.dims[l][0], fy = M.dims[l][1], fz = M.dims[l][2];
    const int shx = M.shift[l][0], shy = M.shift[l][1], shz = M.shift[l][2];
    bool any = false;
    for (int c = 0; c < (1 << (shx + (D == 3 ? shy : 0) + shz)); ++c) {
        const int bx = c & ((1 << shx) - 1);
        const int by = D == 3 ? (c >> shx) & ((1 << shy) - 1) : 0;
        const int bz = c >> (shx + (D == 3 ? shy : 0));
        const int ax = (px << shx) + bx;
        const int ay = D == 3 ? (py << shy) + by : 0;
        const int az = (pz << shz) + bz;
        if (ax >= fx || ay >= fy || az >= fz) continue;
        const int If = (az * fy + ay) * fx + ax;
        if (vf[If] == 0.f) continue;          // inactive node
        any = true;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = (D == 3 ? -1 : 0); dy <= (D == 3 ? 1 : 0); ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const float aval = Af[(int64_t)stencil_index<D>(dx, dy, dz) * Nf + If];
                    if (aval == 0.f) continue;
                    const int jx = ax + dx, jy = ay + dy, jz = az + dz;
                    stencil_add<S>(acc, stencil_index<D>((jx >> shx) - px, D == 3 ? (jy >> shy) - py : 0,
                                                         (jz >> shz) - pz), aval);
                }
    }
    float *Ac = W.mg_pool + M.offA[l + 1];
    float *vc = W.mg_pool + M.offv[l + 1];
#pragma unroll
    for (int o = 0; o < S; ++o) Ac[(int64_t)o * Nc + Ic] = acc[o];
    const float cc = acc[stencil_index<D>(0, 0, 0)];
    vc[Ic] = (any && cc != 0.f) ? 1.f / cc : 0.f;
}

template <int D>
__device__ __forceinline__ void mg_coarsen_body(const Work &W, const MG &M, int l, int bid_)
{
    if (step_failed(W.status)) return;
    const int Ic = bid_ * blockDim.x + threadIdx.x;
    if (Ic < M.n[l + 1]) coarsen_node<D>(W, M, l, Ic);
}

template <int D>
__global__ void k_mg_coarsen(Work W, MG M, int l)
{
    mg_coarsen_body<D>(W, M, l, blockIdx.x);
}

// Levels l0+1 .. L (small) built by one block, level after level.
template <int D>
__device__ __forceinline__ void mg_coarsen_small_body(const Work &W, const MG &M, int l0, int bid_)
{
    if (step_failed(W.status)) return;
    for (int l = l0; l < M.L; ++l) {
        for (int Ic = threadIdx.x; Ic < M.n[l + 1]; Ic += blockDim.x) coarsen_node<D>(W, M, l, Ic);
        __threadfence_block();
        __syncthreads();
    }
}

template <int D>
__global__ void k_mg_coarsen_small(Work W, MG M, int l0)
{
    mg_coarsen_small_body<D>(W, M, l0, blockIdx.x);
}

__device__ __forceinline__ void mg_dsc_body(const Work &W, int n, int bid_)
{
    if (step_failed(W.status)) return;
    int i = bid_ * blockDim.x + threadIdx.x;
    if (i >= n) return;
    W.mg_dsc[i] = (W.pcnt[i] >= 0 && W.diag[i] != 0.0) ? (float)(1.0 / W.diag[i]) : 0.f;
}

__global__ void k_mg_dsc(Work W, int n)
{
    mg_dsc_body(W, n, blockIdx.x);
}

// The large-system solve iterates over the unknown rows only (walls, virtual
// and free-surface particles have no row): their ascending list, by a scan.
__device__ __forceinline__ void urow_flags_body(const Work &W, int n, int bid_)
{
    if (step_failed(W.status)) return;
    const int i = bid_ * blockDim.x + threadIdx.x;
    if (i < n) W.urow_flag[i] = W.pcnt[i] >= 0 ? 1 : 0;
}

__global__ void k_urow_flags(Work W, int n)
{
    urow_flags_body(W, n, blockIdx.x);
}

__device__ __forceinline__ void urow_scatter_body(const Work &W, int n, int bid_)
{
    if (step_failed(W.status)) return;
    const int i = bid_ * blockDim.x + threadIdx.x;
    if (i < n && W.urow_flag[i]) W.urow[W.urow_pos[i]] = i;
}

__global__ void k_urow_scatter(Work W, int n)
{
    urow_scatter_body(W, n, blockIdx.x);
}

// coarse levels up to this size are built by one block (2-D wave, set-up per step
// by the threshold: 4096 nodes 88 us, 2048 57, 1100 57, 512 55, 256 61; VCT_MG_SMALL
// overrides)
constexpr int SMALL_LEVEL = 1024;
static int small_level()
{
    static const int v = getenv("VCT_MG_SMALL") ? atoi(getenv("VCT_MG_SMALL")) : SMALL_LEVEL;
    return v;
}

void launch_mg_setup(const DevParams &P, Work W, const MG &M, int64_t n, cudaStream_t st,
                     bool rows_list)
{
    if (rows_list) {
        k_urow_flags<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(W, (int)n);
        exclusive_scan<int32_t>(W.urow_flag, W.urow_pos, W.scan_tmp, n, st);
        k_urow_scatter<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(W, (int)n);
    }
    k_mg_dsc<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(W, (int)n);
    const unsigned g1 = (unsigned)(((int64_t)M.n[1] * 32 + 255) / 256);   // a warp per cell
    const int mixed = P.precision == VCT_MIXED;
    if (mg_rowcell_on(M)) {   // a row group per row, then level 1 from its cell sums
        const unsigned gr = (unsigned)((n * (P.dim == 2 ? 4 : 8) + 255) / 256);
        const unsigned gl = (unsigned)(((int64_t)M.n[1] + 255) / 256);
        if (P.dim == 2) {
            k_mg_rowcell<2><<<gr, 256, 0, st>>>(W, M, (int)n, mixed);
            k_mg_level1_rc<2><<<gl, 256, 0, st>>>(W, M);
        } else {
            k_mg_rowcell<3><<<gr, 256, 0, st>>>(W, M, (int)n, mixed);
            k_mg_level1_rc<3><<<gl, 256, 0, st>>>(W, M);
        }
    } else {
        if (P.dim == 2) k_mg_level1<2><<<g1, 256, 0, st>>>(W, M, mixed);
        else k_mg_level1<3><<<g1, 256, 0, st>>>(W, M, mixed);
    }
    int l = 1;
    for (; l < M.L && M.n[l + 1] > small_level(); ++l) {
        const unsigned g = (unsigned)((M.n[l + 1] + 127) / 128);
        if (P.dim == 2) k_mg_coarsen<2><<<g, 128, 0, st>>>(W, M, l);
        else k_mg_coarsen<3><<<g, 128, 0, st>>>(W, M, l);
    }
    if (l < M.L) {
        if (P.dim == 2) k_mg_coarsen_small<2><<<1, 256, 0, st>>>(W, M, l);
        else k_mg_coarsen_small<3><<<1, 256, 0, st>>>(W, M, l);
    }
}

bool mg_rowcell_on(const MG &M)
{
    return M.rowcell != 0 && M.fly == 0;
}

int mg_setup_launches(const MG &M)
{
    int l = 1, n = mg_rowcell_on(M) ? 3 : 2;   // dsc, (row-cell operator,) level 1
    for (; l < M.L && M.n[l + 1] > small_level(); ++l) ++n;
    return n + (l < M.L ? 1 : 0);
}

// A view of one coarse level: its stencil operator (entry-major, S entries per
// node) and the vectors dinv, b, z, zu -- in global memory for the grid-wide
// phases (data written by other blocks read with __ldcg), or in block 0's
// shared memory for the small levels.
struct LV {
    const float *A;
    float *dinv, *b, *z, *zu;
    int n, nx, ny, nz;
    int shx, shy, shz;   // coarsening shifts from this level to the next
};

__device__ __forceinline__ LV lv_global(const Work &W, const MG &M, int l)
{
    LV v;
    const int n = M.n[l];
    float *base = W.mg_pool + M.offv[l];
    v.A = W.mg_pool + M.offA[l];
    v.dinv = base;
    v.b = base + n;
    v.z = base + 2 * n;
    v.zu = base + 3 * n;
    v.n = n;
    v.nx = M.dims[l][0];
    v.ny = M.dims[l][1];
    v.nz = M.dims[l][2];
    v.shx = M.shift[l][0];
    v.shy = M.shift[l][1];
    v.shz = M.shift[l][2];
    return v;
}

__device__ __forceinline__ LV lv_shared(float *sh, const MG &M, int l)
{
    LV v;
    const int n = M.n[l];
    float *base = sh + M.soff[l];
    v.A = base;
    v.dinv = base + (long long)M.S * n;
    v.b = v.dinv + n;
    v.z = v.b + n;
    v.zu = v.z + n;
    v.n = n;
    v.nx = M.dims[l][0];
    v.ny = M.dims[l][1];
    v.nz = M.dims[l][2];
    v.shx = M.shift[l][0];
    v.shy = M.shift[l][1];
    v.shz = M.shift[l][2];
    return v;
}

template <bool GL>
__device__ __forceinline__ float ldv(const float *p)
{
    if (GL) return __ldcg(p);
    return *p;
}

// Down phase: nodes of the coarse level c sum the residuals of their children
// in f and take one damped Jacobi step from zero.  The G = 2^(shifts) children
// of a coarse node (2, 4 or 8) are the lanes of one group of G consecutive
// lanes, each lane one child's residual, summed across the group by shuffles
// in a fixed order: G x (coarse nodes) threads share the work instead of one
// thread per coarse node walking its children (measured on the 3-D slice: a
// level's down phase 65.6 -> 17.1 us on average).  start and stride are
// multiples of 32, so a group
// never straddles a warp and its lanes always run the same trips.
template <int D, bool GL>
__device__ void lv_down(const LV &f, const LV &c, float om, int start, int stride)
{
    const int sy = D == 3 ? f.shy : 0;
    const int lg2 = f.shx + sy + f.shz;
    const int G = 1 << lg2;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned gmask = G >= 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(unsigned)(G - 1)));
    const long long total = (long long)c.n << lg2;
    for (long long q = start; q < total; q += stride) {
        const int Ic = (int)(q >> lg2), ch = (int)(q & (G - 1));
        const int px = Ic % c.nx, pr = Ic / c.nx, py = pr % c.ny, pz = pr / c.ny;
        const int ax = (px << f.shx) + (ch & ((1 << f.shx) - 1));
        const int ay = D == 3 ? (py << f.shy) + ((ch >> f.shx) & ((1 << f.shy) - 1)) : 0;
        const int az = (pz << f.shz) + (ch >> (f.shx + sy));
        float res = 0.f;
        if (ax < f.nx && ay < f.ny && az < f.nz) {
            const int If = (az * f.ny + ay) * f.nx + ax;
            if (f.dinv[If] != 0.f) {
                res = ldv<GL>(f.b + If);
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = (D == 3 ? -1 : 0); dy <= (D == 3 ? 1 : 0); ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            const int jx = ax + dx, jy = ay + dy, jz = az + dz;
                            if (jx < 0 || jy < 0 || jz < 0 || jx >= f.nx || jy >= f.ny || jz >= f.nz) continue;
                            res -= f.A[(int64_t)stencil_index<D>(dx, dy, dz) * f.n + If] *
                                   ldv<GL>(f.z + (jz * f.ny + jy) * f.nx + jx);
                        }
            }
        }
        for (int o = G >> 1; o > 0; o >>= 1) res += __shfl_xor_sync(gmask, res, o, G);
        if (ch == 0) {
            c.b[Ic] = res;
            c.z[Ic] = om * res * c.dinv[Ic];
        }
    }
}

// Up phase: nodes of f add kappa x the coarse correction (c.zu) and take one
// damped Jacobi step; the result goes to f.zu.
template <int D, bool GL>
__device__ void lv_up(const LV &f, const LV &c, float om, float kap, int start, int stride)
{
    for (int I = start; I < f.n; I += stride) {
        const float dinv = f.dinv[I];
        if (dinv == 0.f) {
            f.zu[I] = 0.f;
            continue;
        }
        const int cx = I % f.nx, cr = I / f.nx, cy = cr % f.ny, cz = cr / f.ny;
        float res = ldv<GL>(f.b + I), zi = 0.f;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = (D == 3 ? -1 : 0); dy <= (D == 3 ? 1 : 0); ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int jx = cx + dx, jy = cy + dy, jz = cz + dz;
                    if (jx < 0 || jy < 0 || jz < 0 || jx >= f.nx || jy >= f.ny || jz >= f.nz) continue;
                    const int J = (jz * f.ny + jy) * f.nx + jx;
                    const int Jc = ((jz >> f.shz) * c.ny + (D == 3 ? (jy >> f.shy) : 0)) * c.nx + (jx >> f.shx);
                    const float zj = ldv<GL>(f.z + J) + kap * ldv<GL>(c.zu + Jc);
                    if (dx == 0 && dy == 0 && dz == 0) zi = zj;
                    res -= f.A[(int64_t)stencil_index<D>(dx, dy, dz) * f.n + I] * zj;
                }
        f.zu[I] = zi + om * dinv * res;
    }
}

// Coarsest level in block 0's shared memory: Jacobi sweeps from z; result in zu.
template <int D>
__device__ void lv_coarsest(const LV &c, float om, int sweeps)
{
    for (int sw = 0; sw < sweeps; ++sw) {
        const float *src = (sw & 1) ? c.zu : c.z;
        float *dst = (sw & 1) ? c.z : c.zu;
        for (int I = threadIdx.x; I < c.n; I += blockDim.x) {
            const float dinv = c.dinv[I];
            if (dinv == 0.f) {
                dst[I] = 0.f;
                continue;
            }
            const int cx = I % c.nx, cr = I / c.nx, cy = cr % c.ny, cz = cr / c.ny;
            float res = c.b[I];
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = (D == 3 ? -1 : 0); dy <= (D == 3 ? 1 : 0); ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int jx = cx + dx, jy = cy + dy, jz = cz + dz;
                        if (jx < 0 || jy < 0 || jz < 0 || jx >= c.nx || jy >= c.ny || jz >= c.nz) continue;
                        res -= c.A[(int64_t)stencil_index<D>(dx, dy, dz) * c.n + I] *
                               src[(jz * c.ny + jy) * c.nx + jx];
                    }
            dst[I] = src[I] + om * dinv * res;
        }
        __syncthreads();
    }
    if (!(sweeps & 1)) {
        for (int I = threadIdx.x; I < c.n; I += blockDim.x) c.zu[I] = c.z[I];
        __syncthreads();
    }
}

// Block 0 copies the operators and dinv of the shared-memory levels once per solve.
__device__ void mg_load_shared(const Work &W, const MG &M, float *sh)
{
    for (int l = M.first_local; l <= M.L; ++l) {
        const LV g = lv_global(W, M, l), s = lv_shared(sh, M, l);
        const long long na = (long long)M.S * g.n;
        float *As = (float *)s.A;
        for (long long q = threadIdx.x; q < na; q += blockDim.x) As[q] = g.A[q];
        for (int q = threadIdx.x; q < g.n; q += blockDim.x) s.dinv[q] = g.dinv[q];
    }
    __syncthreads();
}

// Software-pipelined row products (large systems).  Every lane stages the next
// row's count, columns and coefficients (its own slots lg, lg+G, ... below NS*G)
// in shared memory with cp.async while it gathers for the current row (ROW_STAGES
// rows in flight per group), so a row costs about one round trip (the gathers)
// instead of three (count, operator, gathers).  Each thread reads back only
// what it copied itself, so cp.async.wait_group alone orders the copies before
// the reads.  The staging area is slot-major over the block's threads.
template <int B>
__device__ __forceinline__ void cp_async(void *sdst, const void *gsrc)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gsrc), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename CT>
__device__ __forceinline__ const CT *coef_ptr(const Work &W);
template <>
__device__ __forceinline__ const double *coef_ptr<double>(const Work &W) { return W.pval; }
template <>
__device__ __forceinline__ const float *coef_ptr<float>(const Work &W) { return W.pvalf; }

#ifndef VCT_ROW_STAGES
#define VCT_ROW_STAGES 2
#endif
constexpr int ROW_STAGES = VCT_ROW_STAGES;
// Slots of a row each lane of a 3-D row group (8 lanes) loads before the row's
// count is known, and stages in the large-system form: 8 x NS3 slots cover a
// row without a second round trip (3-D rows hold ~57-66 coefficients; measured
// on the 2.1M-particle beach, solve per step: 7 slots 90.8 ms, 8 86.8, 9 85.2)
#ifndef VCT_NS3
#define VCT_NS3 9
#endif
constexpr int NS3 = VCT_NS3;

template <typename CT, int NS>
struct RowStage {
    int32_t *pc;   // [ROW_STAGES][KT]
    int32_t *jj;   // [ROW_STAGES][NS][KT]
    CT *aa;        // [ROW_STAGES][NS][KT]
};

template <typename CT, int NS>
__host__ __device__ constexpr size_t row_stage_bytes()
{
    return (size_t)ROW_STAGES * KT * (sizeof(int32_t) * (1 + NS) + sizeof(CT) * NS);
}

// Fine-vector gathers: through L1 (valid after the grid barrier's acquire) or L2 only.
template <typename T>
__device__ __forceinline__ T ldx(const T *p, int j, bool l1)
{
    return l1 ? p[j] : __ldcg(p + j);
}

template <typename CT, int NS>
__device__ __forceinline__ RowStage<CT, NS> row_stage(unsigned char *base, bool staged)
{
    RowStage<CT, NS> S;
    if (!staged) {
        S.aa = nullptr;
        S.jj = S.pc = nullptr;
        return S;
    }
    S.aa = (CT *)base;                                   // 8-byte aligned first
    S.jj = (int32_t *)(base + sizeof(CT) * ROW_STAGES * NS * KT);
    S.pc = S.jj + ROW_STAGES * NS * KT;
    return S;
}

template <typename CT, int G, int NS>
__device__ __forceinline__ void stage_row(const Work &W, const RowStage<CT, NS> &S, int b, int i, int lg)
{
    const int t = threadIdx.x;
    const int64_t cap = W.cap;
    const CT *cv = coef_ptr<CT>(W);
    cp_async<4>(S.pc + b * KT + t, W.pcnt + i);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int kk = lg + s * G;
        if (kk < W.max_nbr) {
            const int64_t q = ell_at<G>(kk, i, cap);
            cp_async<4>(S.jj + (b * NS + s) * KT + t, W.pcol + q);
            cp_async<(int)sizeof(CT)>(S.aa + (b * NS + s) * KT + t, cv + q);
        }
    }
}

// Row operands the epilogue needs besides the product (loaded with the gathers).
template <typename A>
struct Own4 {
    A v[4];
};

// body(i, sum, o) runs for every unknown row i (pcnt >= 0) with the group's sum
// of a_ik x_k over the stored coefficients (the diagonal is not included) and
// o = own(i), whose loads are issued before the gathers so that both share one
// round trip.
// Rows are rows[0..nr) (the unknown rows in ascending order); each row's index
// is loaded one row ahead of its staging, so the list adds no round trip.
template <typename T, typename CT, int G, int NS, typename GetX, typename OwnF, typename Body>
__device__ __forceinline__ void rows_pipelined(const Work &W, const RowStage<CT, NS> &S,
                                               const int32_t *rows, int nr, int g0,
                                               int ngroups, int lg, GetX getx, OwnF own, Body body)
{
    const int t = threadIdx.x;
    const int64_t cap = W.cap;
    if (S.pc == nullptr) {   // staging off: count and operator, then the gathers
        for (int q = g0; q < nr; q += ngroups) {
            const int i = __ldg(rows + q);
            int pc;
            const auto o = own(i);
            T acc = row_dot_pc<T, CT, G, NS>(W, i, lg, pc, getx);
            if (pc < 0) continue;
            acc = group_sum<G>(acc);
            body(i, acc, o);
        }
        return;
    }
    constexpr int R = ROW_STAGES;
    static_assert(R >= 2 && R <= 4, "2 to 4 row stages");
    // iq[k]: index of row q + k ngroups.  At the top of an iteration rows q ..
    // q + (R - 2) ngroups are staged (stages b, b + 1, ... mod R); row
    // q + (R - 1) ngroups is staged now and the index R rows ahead loaded, so
    // the list adds no round trip.
    int iq[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int qk = g0 + k * ngroups;
        iq[k] = qk < nr ? __ldg(rows + qk) : 0;
    }
#pragma unroll
    for (int k = 0; k < R - 1; ++k) {
        if (g0 + k * ngroups < nr) stage_row<CT, G, NS>(W, S, k, iq[k], lg);
        cp_async_commit();
    }
    int b = 0;   // stage of the current row
    for (int q = g0; q < nr; q += ngroups) {
        const int i = iq[0];
        const int bs = b + R - 1 >= R ? b - 1 : b + R - 1;
        if (q + (R - 1) * ngroups < nr) stage_row<CT, G, NS>(W, S, bs, iq[R - 1], lg);
        cp_async_commit();
        const int iafter = q + R * ngroups < nr ? __ldg(rows + q + R * ngroups) : 0;
        cp_async_wait<R - 1>();
        const int pc = S.pc[b * KT + t];
        const auto o = own(i);
        T acc = T(0);
#pragma unroll
        for (int s = 0; s < NS; ++s)
            if (lg + s * G < pc)
                acc += (T)S.aa[(b * NS + s) * KT + t] * getx(S.jj[(b * NS + s) * KT + t]);
        for (int kk = lg + NS * G; kk < pc; kk += G) {
            const int64_t q = ell_at<G>(kk, i, cap);
            acc += (T)coef<CT>(W, q) * getx(W.pcol[q]);
        }
        b = b + 1 == R ? 0 : b + 1;
#pragma unroll
        for (int k = 0; k < R - 1; ++k) iq[k] = iq[k + 1];
        iq[R - 1] = iafter;
        if (pc < 0) continue;
        acc = group_sum<G>(acc);
        body(i, acc, o);
    }
    cp_async_wait<0>();
}

// z_out = M^-1 v.  V(1,1) (M.rowcell = 0): on entry v and z0 = omega D^-1 v
// (the first Jacobi step from zero) are in memory for every unknown row and
// visible grid-wide; each fine product gathers one value per neighbour.
// V(0,1) (M.rowcell = 1): v alone; the cells take the restriction of v, and the
// fine post-smoothing reads the row-cell operator W.mg_B and the cells'
// correction instead of the rows' coefficients (z0, zb unused).  Returns false
// if a grid barrier timed out.
template <typename T, typename CT, int G, int NS, int D>
__device__ bool vcycle(const Work &W, const MG &M, float *sh, const RowStage<CT, NS> &S, int n,
                       const T *v, const T *z0, T *zb, T *zout, int lg, bool lead, int g0, int ngroups,
                       int gtid, int gthreads, unsigned vb, unsigned vnb)
{
    const unsigned nb = vnb;
    const float om = M.omega, kap = M.kappa;
    const bool l1 = M.gather_l1 != 0;
    const bool rc = M.rowcell != 0;
    const int32_t *urow = W.urow;
    const int nu = W.urow_pos[n];
    T *r0 = (T *)W.kr0;
    if (!rc) {
        // D0: fine residual r0 = v - A z0
        rows_pipelined<T, CT, G, NS>(W, S, urow, nu, g0, ngroups, lg, [&](int j) { return ldx(z0, j, l1); },
            [&](int i) { return Own4<T>{{__ldcg(v + i), __ldcg(z0 + i), (T)W.diag[i], T(0)}}; },
            [&](int i, T acc, const Own4<T> &o) {
                if (lead) r0[i] = o.v[0] - acc - o.v[2] * o.v[1];
            });
        if (!grid_barrier(W.bar, nb, W.status, vb, W.spin_limit)) return false;
    }
    // D1: restriction to the cells (of r0, or of v in V(0,1)), one Jacobi step
    // from zero on level 1
    {
        const LV c = lv_global(W, M, 1);
        const T *rs = rc ? v : r0;
        for (int I = gtid; I < c.n; I += gthreads) {
            float bs = 0.f;
            const int a = W.cell_start[I], b = W.cell_start[I + 1];
            for (int i = a; i < b; ++i)
                if (W.pcnt[i] >= 0) bs += (float)__ldcg(rs + i);
            c.b[I] = bs;
            c.z[I] = M.omega_c * bs * c.dinv[I];
        }
    }
    if (!grid_barrier(W.bar, nb, W.status, vb, W.spin_limit)) return false;
    const int fl = M.first_local;
    for (int l = 1; l < fl; ++l) {
        lv_down<D, true>(lv_global(W, M, l), lv_global(W, M, l + 1), M.omega_c, gtid, gthreads);
        if (!grid_barrier(W.bar, nb, W.status, vb, W.spin_limit)) return false;
    }
    if (vb == 0) {
        {
            const LV g = lv_global(W, M, fl), s = lv_shared(sh, M, fl);
            for (int q = threadIdx.x; q < g.n; q += blockDim.x) {
                s.b[q] = __ldcg(g.b + q);
                s.z[q] = __ldcg(g.z + q);
            }
            __syncthreads();
        }
        for (int l = fl; l < M.L; ++l) {
            lv_down<D, false>(lv_shared(sh, M, l), lv_shared(sh, M, l + 1), M.omega_c, threadIdx.x, blockDim.x);
            __syncthreads();
        }
        lv_coarsest<D>(lv_shared(sh, M, M.L), M.omega_c, M.coarse_sweeps);
        for (int l = M.L - 1; l >= fl; --l) {
            lv_up<D, false>(lv_shared(sh, M, l), lv_shared(sh, M, l + 1), M.omega_c, M.kappa_c, threadIdx.x, blockDim.x);
            __syncthreads();
        }
        {
            const LV g = lv_global(W, M, fl), s = lv_shared(sh, M, fl);
            for (int q = threadIdx.x; q < g.n; q += blockDim.x) g.zu[q] = s.zu[q];
        }
    }
    if (!grid_barrier(W.bar, nb, W.status, vb, W.spin_limit)) return false;
    for (int l = fl - 1; l >= 1; --l) {
        lv_up<D, true>(lv_global(W, M, l), lv_global(W, M, l + 1), M.omega_c, M.kappa_c, gtid, gthreads);
        if (!grid_barrier(W.bar, nb, W.status, vb, W.spin_limit)) return false;
    }
    if (rc) {
        // U0 of V(0,1): zb = kappa zu_1(cell) and one damped Jacobi step,
        // z = zb + omega D^-1 (v - A zb) with (A zb)_i = kappa sum_o B[o][i] zu_1(cell(i) + o)
        const float *zu1 = W.mg_pool + M.offv[1] + 3 * M.n[1];
        const int nx = M.dims[1][0], ny = M.dims[1][1], nz = M.dims[1][2];
        const int64_t cap = W.cap;
        const float *B = W.mg_B;
        for (int q = gtid; q < nu; q += gthreads) {
            const int i = __ldg(urow + q);
            const int I = W.cellid[i];
            int cx, cy, cz;
            mg_coords(M, 1, I, cx, cy, cz);
            float acc = 0.f;
#pragma unroll
            for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
                for (int dy = (D == 3 ? -1 : 0); dy <= (D == 3 ? 1 : 0); ++dy)
#pragma unroll
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int jx = cx + dx, jy = cy + dy, jz = cz + dz;
                        if (jx < 0 || jx >= nx || jy < 0 || jy >= ny || jz < 0 || jz >= nz) continue;
                        acc += __ldg(B + (int64_t)stencil_index<D>(dx, dy, dz) * cap + i) *
                               __ldcg(zu1 + (jz * ny + jy) * nx + jx);
                    }
            const T zi = (T)kap * (T)__ldcg(zu1 + I);
            const T res = __ldcg(v + i) - (T)kap * (T)acc;
            zout[i] = zi + (T)om * res * (T)W.mg_dsc[i];
        }
        return grid_barrier(W.bar, nb, W.status, vb, W.spin_limit);
    }
    // P0: prolongation from the cells, zb = z0 + kappa zu_1(cell)
    {
        const float *zu1 = W.mg_pool + M.offv[1] + 3 * M.n[1];
        for (int q = gtid; q < nu; q += gthreads) {
            const int i = __ldg(urow + q);
            zb[i] = __ldcg(z0 + i) + (T)kap * (T)__ldcg(zu1 + W.cellid[i]);
        }
    }
    if (!grid_barrier(W.bar, nb, W.status, vb, W.spin_limit)) return false;
    // U0: one damped Jacobi step on the fine level
    rows_pipelined<T, CT, G, NS>(W, S, urow, nu, g0, ngroups, lg, [&](int j) { return ldx(zb, j, l1); },
        [&](int i) { return Own4<T>{{__ldcg(zb + i), __ldcg(v + i), (T)W.diag[i], (T)W.mg_dsc[i]}}; },
        [&](int i, T acc, const Own4<T> &o) {
            if (lead) {
                const T res = o.v[1] - acc - o.v[2] * o.v[0];
                zout[i] = o.v[0] + (T)om * res * o.v[3];
            }
        });
    return grid_barrier(W.bar, nb, W.status, vb, W.spin_limit);
}

// Right-preconditioned BiCGSTAB inside FP64 iterative refinement (as k_krylov).
// The large-system solve on vnb blocks (block vb of them): the whole grid, or
// one scenario's subset of a batched launch.
template <typename T, typename CT, int G, int NS, int D>
__device__ void krylov_explicit_solve(const Work &W, const MG &M, int n, int maxit, double rtol,
                                      double inner_floor, int32_t *iters_out, double *resid_out,
                                      unsigned vb, unsigned vnb)
{
    if (step_failed(W.status)) return;
    const unsigned nb = vnb;
    const int lg = threadIdx.x & (G - 1);
    const bool lead = lg == 0;
    const int ngroups = (int)(vnb * blockDim.x) / G;
    const int g0 = (int)(vb * blockDim.x + threadIdx.x) / G;
    const int gtid = (int)(vb * blockDim.x + threadIdx.x), gthreads = (int)(vnb * blockDim.x);
    extern __shared__ __align__(16) float mg_sh[];
    if (vb == 0) mg_load_shared(W, M, mg_sh);
    const RowStage<CT, NS> S = row_stage<CT, NS>((unsigned char *)mg_sh + M.stage_off, M.staged != 0);
    const int32_t *urow = W.urow;
    const int nu = W.urow_pos[n];
    const bool l1 = M.gather_l1 != 0;
    const bool rc = M.rowcell != 0;
    const float om = M.omega;
    double *x = W.kx, *f = W.kf;
    T *r = (T *)W.kr, *rh = (T *)W.krh, *s = (T *)W.ks, *t = (T *)W.kt, *dl = (T *)W.kd;
    T *pold = (T *)W.kp0, *pnew = (T *)W.kp1, *vold = (T *)W.kv0, *vnew = (T *)W.kv1;
    T *ph = (T *)W.kq0, *sh = (T *)W.kq1;   // p^ = M^-1 p, s^ = M^-1 s
    T *z0 = (T *)W.kz0, *zb = (T *)W.kzb;
    int total_it = 0;
    bool fail = false;
    double bn = 0.0, rn = 0.0;
    for (int outer = 0;; ++outer) {
        double part[2] = {0.0, 0.0};
        rows_pipelined<double, CT, G, NS>(W, S, urow, nu, g0, ngroups, lg, [&](int j) { return ldx(x, j, l1); },
            [&](int i) { return Own4<double>{{W.bvec[i], W.diag[i], __ldcg(x + i), 0.0}}; },
            [&](int i, double ax, const Own4<double> &o) {
                if (lead) {
                    const double bi = o.v[0], fi = bi - (ax + o.v[1] * o.v[2]);
                    f[i] = fi;
                    part[0] += fi * fi;
                    part[1] += bi * bi;
                }
            });
        block_partials<2>(part, W.partial, vb);
        if (!grid_barrier(W.bar, nb, W.status, vb, W.spin_limit)) return;
        double tot[2];
        grid_totals<2>(W.partial, nb, tot);
        rn = sqrt(tot[0]);
        bn = sqrt(tot[1]);
        if (bn == 0.0) {
            for (int i = g0; i < n; i += ngroups)
                if (lead) x[i] = 0.0;
            rn = 0.0;
            break;
        }
        if (rn <= rtol * bn) break;
        if (total_it >= maxit || outer >= 64) {
            fail = true;
            break;
        }
        const double fn = rn, tol_in = fmax(rtol * bn / rn, inner_floor);
        double rho = fn * fn, rho_old = 1.0, alpha = 1.0, omega = 1.0;
        bool first = true, have_pend = false;
        double pend_a = 0.0, pend_w = 0.0;
        for (;;) {
            if (total_it >= maxit) break;
            ++total_it;
            const double beta = first ? 0.0 : (rho / rho_old) * (alpha / omega);
            const T tb = (T)beta, tw = (T)omega, ta = (T)pend_a, twp = (T)pend_w;
            // E1 (own rows): apply the pending update, r = s - w t, p_new = r + beta (p - w v)
            for (int q = gtid; q < nu; q += gthreads) {
                const int i = __ldg(urow + q);
                T ri, pn;
                if (first) {
                    ri = (T)__ldcg(f + i);
                    rh[i] = ri;
                    dl[i] = T(0);
                    pn = ri;
                } else {
                    ri = __ldcg(s + i) - tw * __ldcg(t + i);
                    pn = ri + tb * (pold[i] - tw * __ldcg(vold + i));
                    if (have_pend) dl[i] += ta * __ldcg(ph + i) + twp * __ldcg(sh + i);
                }
                r[i] = ri;
                pnew[i] = pn;
                if (!rc) z0[i] = (T)om * pn * (T)W.mg_dsc[i];
            }
            if (!grid_barrier(W.bar, nb, W.status, vb, W.spin_limit)) return;
            if (!vcycle<T, CT, G, NS, D>(W, M, mg_sh, S, n, pnew, z0, zb, ph, lg, lead, g0, ngroups, gtid, gthreads, vb, vnb))
                return;
            first = false;
            have_pend = false;
            // v = A p^, partial (rh, v)
            T pa = T(0);
            rows_pipelined<T, CT, G, NS>(W, S, urow, nu, g0, ngroups, lg, [&](int j) { return ldx(ph, j, l1); },
                [&](int i) { return Own4<T>{{(T)W.diag[i], __ldcg(ph + i), __ldcg(rh + i), T(0)}}; },
                [&](int i, T acc, const Own4<T> &o) {
                    if (lead) {
                        acc += o.v[0] * o.v[1];
                        vnew[i] = acc;
                        pa += o.v[2] * acc;
                    }
                });
            {
                double pd[1] = {(double)pa};
                block_partials<1>(pd, W.partial, vb);
            }
            if (!grid_barrier(W.bar, nb, W.status, vb, W.spin_limit)) return;
            double tv[1];
            grid_totals<1>(W.partial, nb, tv);
            if (tv[0] == 0.0) {
                fail = true;
                break;
            }
            alpha = rho / tv[0];
            const T ta2 = (T)alpha;
            // E2 (own rows): s = r - alpha v
            for (int q = gtid; q < nu; q += gthreads) {
                const int i = __ldg(urow + q);
                const T si = r[i] - ta2 * __ldcg(vnew + i);
                s[i] = si;
                if (!rc) z0[i] = (T)om * si * (T)W.mg_dsc[i];
            }
            if (!grid_barrier(W.bar, nb, W.status, vb, W.spin_limit)) return;
            if (!vcycle<T, CT, G, NS, D>(W, M, mg_sh, S, n, s, z0, zb, sh, lg, lead, g0, ngroups, gtid, gthreads, vb, vnb))
                return;
            // t = A s^; partials (t,s) (t,t) (s,s) (rh,s) (rh,t)
            T pb0 = T(0), pb1 = T(0), pb2 = T(0), pb3 = T(0), pb4 = T(0);
            rows_pipelined<T, CT, G, NS>(W, S, urow, nu, g0, ngroups, lg, [&](int j) { return ldx(sh, j, l1); },
                [&](int i) { return Own4<T>{{__ldcg(s + i), __ldcg(rh + i), (T)W.diag[i], __ldcg(sh + i)}}; },
                [&](int i, T acc, const Own4<T> &o) {
                    if (lead) {
                        const T si = o.v[0], hi = o.v[1];
                        acc += o.v[2] * o.v[3];
                        t[i] = acc;
                        pb0 += acc * si;
                        pb1 += acc * acc;
                        pb2 += si * si;
                        pb3 += hi * si;
                        pb4 += hi * acc;
                    }
                });
            {
                double pd[5] = {(double)pb0, (double)pb1, (double)pb2, (double)pb3, (double)pb4};
                block_partials<5>(pd, W.partial, vb);
            }
            if (!grid_barrier(W.bar, nb, W.status, vb, W.spin_limit)) return;
            double tq[5];
            grid_totals<5>(W.partial, nb, tq);
            T *tp = pold; pold = pnew; pnew = tp;
            tp = vold; vold = vnew; vnew = tp;
            have_pend = true;
            pend_a = alpha;
            if (sqrt(tq[2]) <= tol_in * fn) {
                pend_w = 0.0;
                break;
            }
            if (tq[1] == 0.0) {
                pend_w = 0.0;
                fail = true;
                break;
            }
            omega = tq[0] / tq[1];
            pend_w = omega;
            rho_old = rho;
            rho = tq[3] - omega * tq[4];
            const double rr = tq[2] - 2.0 * omega * tq[0] + omega * omega * tq[1];
            if (sqrt(fmax(rr, 0.0)) <= tol_in * fn || rho == 0.0) break;
        }
        const T fa = (T)pend_a, fw = (T)pend_w;
        for (int q = gtid; q < nu; q += gthreads) {
            const int i = __ldg(urow + q);
            T d = dl[i];
            if (have_pend) d += fa * __ldcg(ph + i) + fw * __ldcg(sh + i);
            x[i] += (double)d;
        }
        if (!grid_barrier(W.bar, nb, W.status, vb, W.spin_limit)) return;
        if (fail) break;
    }
    if (vb == 0 && threadIdx.x == 0) {
        if (fail) set_error(W.status, VCT_ERR_NOCONV, -1);
        iters_out[0] += total_it;
        if (total_it > iters_out[1]) iters_out[1] = total_it;
        iters_out[2] = total_it;
        *resid_out = bn > 0.0 ? rn / bn : 0.0;
    }
}

template <typename T, typename CT, int G, int NS, int D>
__global__ void __launch_bounds__(KT, VCT_KMG_MINB) k_krylov_mg(Work W, MG M, int n, int maxit, double rtol,
                                                  double inner_floor, int32_t *iters_out,
                                                  double *resid_out)
{
    krylov_explicit_solve<T, CT, G, NS, D>(W, M, n, maxit, rtol, inner_floor, iters_out, resid_out,
                                           blockIdx.x, gridDim.x);
}

// z_out = M^-1 v for the fine vector given on the fly by in(j).  own(i) runs once
// for every unknown row in the first phase (lane 0 of the row's group, or the
// cell's thread without pre-smoothing), before any phase writes z_out; it must
// not write what in(j) reads.  Returns false if a grid barrier timed out.
template <typename T, typename CT, int G, int NS, int D, typename In, typename Own>
__device__ bool vcycle_fly(const Work &W, const MG &M, float *sh, int n, In in, Own own, T *zout,
                       int lg, bool lead, int g0, int ngroups, int gtid, int gthreads, unsigned vb,
                       unsigned vnb)
{
    const unsigned nb = vnb;
    const float om = M.omega, kap = M.kappa;
    T *r0 = (T *)W.kr0;
    const bool pre = M.presmooth != 0;
    // D0 (V(1,1) only): fine residual of one Jacobi step from zero, r0 = v - A (om D^-1 v)
    if (pre) {
    for (int i = g0; i < n; i += ngroups) {
        int pc;
        T acc = row_dot_pc<T, CT, G, NS>(W, i, lg, pc, [&](int j) {
            return (T)om * in(j) * (T)__ldcg(W.mg_dsc + j);
        });
        if (pc < 0) continue;
        acc = group_sum<G>(acc);
        if (lead) {
            own(i);
            const T vi = in(i);
            r0[i] = vi - acc - (T)om * vi;
        }
    }
    if (!grid_barrier(W.bar, nb, W.status, vb, W.spin_limit)) return false;
    }
    // D1: restriction to the cells (of r0, or of v itself without pre-smoothing,
    // where own(i) runs here instead), one Jacobi step from zero on level 1
    {
        const LV c = lv_global(W, M, 1);
        for (int I = gtid; I < c.n; I += gthreads) {
            float bs = 0.f;
            const int a = W.cell_start[I], b = W.cell_start[I + 1];
            for (int i = a; i < b; ++i) {
                if (W.pcnt[i] < 0) continue;
                if (pre) {
                    bs += (float)__ldcg(r0 + i);
                } else {
                    own(i);
                    bs += (float)in(i);
                }
            }
            c.b[I] = bs;
            c.z[I] = M.omega_c * bs * c.dinv[I];
        }
    }
    if (!grid_barrier(W.bar, nb, W.status, vb, W.spin_limit)) return false;
    const int fl = M.first_local;
    for (int l = 1; l < fl; ++l) {
        lv_down<D, true>(lv_global(W, M, l), lv_global(W, M, l + 1), M.omega_c, gtid, gthreads);
        if (!grid_barrier(W.bar, nb, W.status, vb, W.spin_limit)) return false;
    }
    if (vb == 0) {
        // levels fl..L in shared memory: b and z of level fl come from global
        {
            const LV g = lv_global(W, M, fl), s = lv_shared(sh, M, fl);
            for (int q = threadIdx.x; q < g.n; q += blockDim.x) {
                s.b[q] = __ldcg(g.b + q);
                s.z[q] = __ldcg(g.z + q);
            }
            __syncthreads();
        }
        for (int l = fl; l < M.L; ++l) {
            lv_down<D, false>(lv_shared(sh, M, l), lv_shared(sh, M, l + 1), M.omega_c, threadIdx.x, blockDim.x);
            __syncthreads();
        }
        lv_coarsest<D>(lv_shared(sh, M, M.L), M.omega_c, M.coarse_sweeps);
        for (int l = M.L - 1; l >= fl; --l) {
            lv_up<D, false>(lv_shared(sh, M, l), lv_shared(sh, M, l + 1), M.omega_c, M.kappa_c, threadIdx.x, blockDim.x);
            __syncthreads();
        }
        {
            const LV g = lv_global(W, M, fl), s = lv_shared(sh, M, fl);
            for (int q = threadIdx.x; q < g.n; q += blockDim.x) g.zu[q] = s.zu[q];
        }
    }
    if (!grid_barrier(W.bar, nb, W.status, vb, W.spin_limit)) return false;
    for (int l = fl - 1; l >= 1; --l) {
        lv_up<D, true>(lv_global(W, M, l), lv_global(W, M, l + 1), M.omega_c, M.kappa_c, gtid, gthreads);
        if (!grid_barrier(W.bar, nb, W.status, vb, W.spin_limit)) return false;
    }
    // U0: prolongation from the cells + one damped Jacobi step on the fine level
    const float *zu1 = W.mg_pool + M.offv[1] + 3 * M.n[1];
    auto zb = [&](int j) -> T {
        const T zc = (T)kap * (T)__ldcg(zu1 + W.cellid[j]);
        return pre ? (T)om * in(j) * (T)__ldcg(W.mg_dsc + j) + zc : zc;
    };
    for (int i = g0; i < n; i += ngroups) {
        int pc;
        T acc = row_dot_pc<T, CT, G, NS>(W, i, lg, pc, zb);
        if (pc < 0) continue;
        acc = group_sum<G>(acc);
        if (lead) {
            const T zi = zb(i);
            const T res = in(i) - acc - (T)W.diag[i] * zi;
            zout[i] = zi + (T)om * res * (T)W.mg_dsc[i];
        }
    }
    return grid_barrier(W.bar, nb, W.status, vb, W.spin_limit);
}

// Right-preconditioned BiCGSTAB inside FP64 iterative refinement (as k_krylov).
// The solve on vnb blocks (block vb of them) sharing W.bar and W.partial: the
// whole grid, or one scenario's subset of a batched launch.
template <typename T, typename CT, int G, int NS, int D>
__device__ void krylov_fly_solve(const Work &W, const MG &M, int n, int maxit, double rtol,
                                 double inner_floor, int32_t *iters_out, double *resid_out,
                                 unsigned vb, unsigned vnb)
{
    if (step_failed(W.status)) return;
    const unsigned nb = vnb;
    const int lg = threadIdx.x & (G - 1);
    const bool lead = lg == 0;
    const int ngroups = (int)(vnb * blockDim.x) / G;
    const int g0 = (int)(vb * blockDim.x + threadIdx.x) / G;
    const int gtid = (int)(vb * blockDim.x + threadIdx.x), gthreads = (int)(vnb * blockDim.x);
    extern __shared__ float mg_sh[];
    if (vb == 0) mg_load_shared(W, M, mg_sh);
    double *x = W.kx, *f = W.kf;
    T *r = (T *)W.kr, *rh = (T *)W.krh, *s = (T *)W.ks, *t = (T *)W.kt, *dl = (T *)W.kd;
    T *pold = (T *)W.kp0, *pnew = (T *)W.kp1, *vold = (T *)W.kv0, *vnew = (T *)W.kv1;
    T *ph = (T *)W.kq0, *sh = (T *)W.kq1;   // p^ = M^-1 p, s^ = M^-1 s
    int total_it = 0;
    bool fail = false;
    double bn = 0.0, rn = 0.0;
    for (int outer = 0;; ++outer) {
        double part[2] = {0.0, 0.0};
        for (int i = g0; i < n; i += ngroups) {
            int pc;
            double ax = row_dot_pc<double, CT, G, NS>(W, i, lg, pc, [&](int j) { return __ldcg(x + j); });
            if (pc < 0) continue;
            ax = group_sum<G>(ax);
            if (lead) {
                double bi = W.bvec[i], fi = bi - (ax + W.diag[i] * x[i]);
                f[i] = fi;
                part[0] += fi * fi;
                part[1] += bi * bi;
            }
        }
        block_partials<2>(part, W.partial, vb);
        if (!grid_barrier(W.bar, nb, W.status, vb, W.spin_limit)) return;
        double tot[2];
        grid_totals<2>(W.partial, nb, tot);
        rn = sqrt(tot[0]);
        bn = sqrt(tot[1]);
        if (bn == 0.0) {
            for (int i = g0; i < n; i += ngroups)
                if (lead) x[i] = 0.0;
            rn = 0.0;
            break;
        }
        if (rn <= rtol * bn) break;
        if (total_it >= maxit || outer >= 64) {
            fail = true;
            break;
        }
        const double fn = rn, tol_in = fmax(rtol * bn / rn, inner_floor);
        double rho = fn * fn, rho_old = 1.0, alpha = 1.0, omega = 1.0;
        bool first = true, have_pend = false;
        double pend_a = 0.0, pend_w = 0.0;
        for (;;) {
            if (total_it >= maxit) break;
            ++total_it;
            const double beta = first ? 0.0 : (rho / rho_old) * (alpha / omega);
            const T tb = (T)beta, tw = (T)omega, ta = (T)pend_a, twp = (T)pend_w;
            const bool fst = first, hp = have_pend;
            // p_new = r + beta (p - w v) with r = s - w t; p^ = M^-1 p_new
            bool ok;
            if (fst) {
                ok = vcycle_fly<T, CT, G, NS, D>(W, M, mg_sh, n,
                    [&](int j) -> T { return (T)__ldcg(f + j); },
                    [&](int i) { const T ri = (T)f[i]; r[i] = ri; rh[i] = ri; pnew[i] = ri; dl[i] = T(0); },
                    ph, lg, lead, g0, ngroups, gtid, gthreads, vb, vnb);
            } else {
                ok = vcycle_fly<T, CT, G, NS, D>(W, M, mg_sh, n,
                    [&](int j) -> T {
                        return (__ldcg(s + j) - tw * __ldcg(t + j)) + tb * (__ldcg(pold + j) - tw * __ldcg(vold + j));
                    },
                    [&](int i) {
                        const T ri = s[i] - tw * t[i];
                        r[i] = ri;
                        pnew[i] = ri + tb * (pold[i] - tw * vold[i]);
                        if (hp) dl[i] += ta * ph[i] + twp * sh[i];
                    },
                    ph, lg, lead, g0, ngroups, gtid, gthreads, vb, vnb);
            }
            if (!ok) return;
            first = false;
            have_pend = false;
            // v = A p^, partial (rh, v)
            T pa = T(0);
            for (int i = g0; i < n; i += ngroups) {
                int pc;
                T acc = row_dot_pc<T, CT, G, NS>(W, i, lg, pc, [&](int j) { return __ldcg(ph + j); });
                if (pc < 0) continue;
                acc = group_sum<G>(acc);
                if (lead) {
                    acc += (T)W.diag[i] * ph[i];
                    vnew[i] = acc;
                    pa += rh[i] * acc;
                }
            }
            {
                double pd[1] = {(double)pa};
                block_partials<1>(pd, W.partial, vb);
            }
            if (!grid_barrier(W.bar, nb, W.status, vb, W.spin_limit)) return;
            double tv[1];
            grid_totals<1>(W.partial, nb, tv);
            if (tv[0] == 0.0) {
                fail = true;
                break;
            }
            alpha = rho / tv[0];
            const T ta2 = (T)alpha;
            // s = r - alpha v; s^ = M^-1 s
            if (!vcycle_fly<T, CT, G, NS, D>(W, M, mg_sh, n,
                    [&](int j) -> T { return __ldcg(r + j) - ta2 * __ldcg(vnew + j); },
                    [&](int i) { s[i] = r[i] - ta2 * vnew[i]; },
                    sh, lg, lead, g0, ngroups, gtid, gthreads, vb, vnb))
                return;
            // t = A s^; partials (t,s) (t,t) (s,s) (rh,s) (rh,t)
            T pb0 = T(0), pb1 = T(0), pb2 = T(0), pb3 = T(0), pb4 = T(0);
            for (int i = g0; i < n; i += ngroups) {
                int pc;
                T acc = row_dot_pc<T, CT, G, NS>(W, i, lg, pc, [&](int j) { return __ldcg(sh + j); });
                if (pc < 0) continue;
                acc = group_sum<G>(acc);
                if (lead) {
                    const T si = s[i], hi = rh[i];
                    acc += (T)W.diag[i] * sh[i];
                    t[i] = acc;
                    pb0 += acc * si;
                    pb1 += acc * acc;
                    pb2 += si * si;
                    pb3 += hi * si;
                    pb4 += hi * acc;
                }
            }
            {
                double pd[5] = {(double)pb0, (double)pb1, (double)pb2, (double)pb3, (double)pb4};
                block_partials<5>(pd, W.partial, vb);
            }
            if (!grid_barrier(W.bar, nb, W.status, vb, W.spin_limit)) return;
            double tq[5];
            grid_totals<5>(W.partial, nb, tq);
            T *tp = pold; pold = pnew; pnew = tp;
            tp = vold; vold = vnew; vnew = tp;
            have_pend = true;
            pend_a = alpha;
            if (sqrt(tq[2]) <= tol_in * fn) {
                pend_w = 0.0;
                break;
            }
            if (tq[1] == 0.0) {
                pend_w = 0.0;
                fail = true;
                break;
            }
            omega = tq[0] / tq[1];
            pend_w = omega;
            rho_old = rho;
            rho = tq[3] - omega * tq[4];
            const double rr = tq[2] - 2.0 * omega * tq[0] + omega * omega * tq[1];
            if (sqrt(fmax(rr, 0.0)) <= tol_in * fn || rho == 0.0) break;
        }
        const T fa = (T)pend_a, fw = (T)pend_w;
        for (int i = g0; i < n; i += ngroups) {
            if (!lead || W.pcnt[i] < 0) continue;
            T d = dl[i];
            if (have_pend) d += fa * ph[i] + fw * sh[i];
            x[i] += (double)d;
        }
        if (!grid_barrier(W.bar, nb, W.status, vb, W.spin_limit)) return;
        if (fail) break;
    }
    if (vb == 0 && threadIdx.x == 0) {
        if (fail) set_error(W.status, VCT_ERR_NOCONV, -1);
        iters_out[0] += total_it;
        if (total_it > iters_out[1]) iters_out[1] = total_it;
        iters_out[2] = total_it;
        *resid_out = bn > 0.0 ? rn / bn : 0.0;
    }
}

template <typename T, typename CT, int G, int NS, int D>
__global__ void __launch_bounds__(KT) k_krylov_mg_fly(Work W, MG M, int n, int maxit, double rtol,
                                                  double inner_floor, int32_t *iters_out,
                                                  double *resid_out)
{
    krylov_fly_solve<T, CT, G, NS, D>(W, M, n, maxit, rtol, inner_floor, iters_out, resid_out,
                                      blockIdx.x, gridDim.x);
}

// Batched solves (ensembles): job j owns blocks [b0, b0 + nb) of one cooperative
// launch and runs its own solve on them, with its own barrier word, partials,
// multigrid levels and status; the jobs never wait on one another.  A block
// copies its job's descriptors into shared memory once.
static_assert(sizeof(FlyJob) % sizeof(int) == 0, "FlyJob copies as ints");

template <typename T, typename CT, int G, int NS, int D, bool EXPL>
__global__ void __launch_bounds__(KT, EXPL ? VCT_KBATCH_MINB : 2) k_krylov_fly_batch(const FlyJob *jobs, int njobs)
{
    __shared__ __align__(16) FlyJob job;
    __shared__ int jid;
    if (threadIdx.x == 0) {
        int j = 0;
        while (j + 1 < njobs && jobs[j + 1].b0 <= blockIdx.x) ++j;
        jid = j;
    }
    __syncthreads();
    {
        const int *src = (const int *)(jobs + jid);
        int *dst = (int *)&job;
        for (int q = threadIdx.x; q < (int)(sizeof(FlyJob) / sizeof(int)); q += blockDim.x) dst[q] = src[q];
    }
    __syncthreads();
    if (EXPL)
        krylov_explicit_solve<T, CT, G, NS, D>(job.W, job.M, job.n, job.maxit, job.rtol,
                                               job.inner_floor, job.W.kiters, job.W.kresid,
                                               blockIdx.x - job.b0, job.nb);
    else
        krylov_fly_solve<T, CT, G, NS, D>(job.W, job.M, job.n, job.maxit, job.rtol, job.inner_floor,
                                          job.W.kiters, job.W.kresid, blockIdx.x - job.b0, job.nb);
}

// Small systems form the V-cycle inputs on the fly inside the products (fewer
// grid barriers); large systems keep them as vectors, so each fine product
// gathers one value per neighbour.  Crossover measured on B300 (solver time per
// iteration): 2-D between 45k (on the fly 8 % faster) and 100k particles
// (vectors 6 % faster); 3-D at ~36k (equal), vectors 15 % faster at 60k.
constexpr long long FLY_MAX_ROWS_2D = 75000, FLY_MAX_ROWS_3D = 30000;

static const void *krylov_mg_fn(int precision, int dim, bool fly)
{
    if (fly) {
        if (precision == VCT_MIXED)
            return dim == 2 ? (const void *)k_krylov_mg_fly<float, float, 4, 5, 2>
                            : (const void *)k_krylov_mg_fly<float, float, 8, NS3, 3>;
        return dim == 2 ? (const void *)k_krylov_mg_fly<double, double, 4, 5, 2>
                        : (const void *)k_krylov_mg_fly<double, double, 8, NS3, 3>;
    }
    if (precision == VCT_MIXED)
        return dim == 2 ? (const void *)k_krylov_mg<float, float, 4, 5, 2>
                        : (const void *)k_krylov_mg<float, float, 8, NS3, 3>;
    return dim == 2 ? (const void *)k_krylov_mg<double, double, 4, 5, 2>
                    : (const void *)k_krylov_mg<double, double, 8, NS3, 3>;
}

bool krylov_mg_fly_default(long long rows, int dim)
{
    return rows <= (dim == 2 ? FLY_MAX_ROWS_2D : FLY_MAX_ROWS_3D);
}

size_t krylov_mg_stage_bytes(int precision, int dim, bool staged)
{
    if (!staged) return 0;
    if (precision == VCT_MIXED) return dim == 2 ? row_stage_bytes<float, 5>() : row_stage_bytes<float, NS3>();
    return dim == 2 ? row_stage_bytes<double, 5>() : row_stage_bytes<double, NS3>();
}

int krylov_mg_coop_blocks(int precision, int dim, size_t smem, bool fly)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void *fn = krylov_mg_fn(precision, dim, fly);
    // the limit is per kernel, shared by every context: only ever raise it
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess && fa.maxDynamicSharedSizeBytes < (int)smem)
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, KT, smem);
    if (per > 4) per = 4;
    int nb = sms * per;
    return nb < PSTRIDE ? nb : PSTRIDE;
}

int launch_krylov_mg(const DevParams &P, Work W, const MG &M, int64_t n, int nblocks_coop,
                     cudaStream_t st)
{
    int nn = (int)n, maxit = P.max_iter;
    double rtol = P.rtol, floor_ = P.inner_floor;
    int32_t *it_out = W.kiters;
    double *res_out = W.kresid;
    const int G = P.dim == 2 ? 4 : 8;
    int64_t want = (n * G + KT - 1) / KT;
    int nblk = (int)(want < nblocks_coop ? want : nblocks_coop);
    if (nblk < 1) nblk = 1;
    MG Mc = M;
    void *args[] = {(void *)&W, (void *)&Mc, (void *)&nn, (void *)&maxit, (void *)&rtol,
                    (void *)&floor_, (void *)&it_out, (void *)&res_out};
    cudaMemsetAsync(W.bar, 0, 2 * sizeof(unsigned int), st);
    cudaError_t e = cudaLaunchCooperativeKernel(krylov_mg_fn(P.precision, P.dim, M.fly != 0),
                                                dim3(nblk), dim3(KT), args, (size_t)M.smem_bytes, st);
    return e == cudaSuccess ? 0 : (int)e;
}

template <bool EXPL>
static const void *krylov_batch_fn_form(int precision, int dim)
{
    if (precision == VCT_MIXED)
        return dim == 2 ? (const void *)k_krylov_fly_batch<float, float, 4, 5, 2, EXPL>
                        : (const void *)k_krylov_fly_batch<float, float, 8, NS3, 3, EXPL>;
    return dim == 2 ? (const void *)k_krylov_fly_batch<double, double, 4, 5, 2, EXPL>
                    : (const void *)k_krylov_fly_batch<double, double, 8, NS3, 3, EXPL>;
}

static const void *krylov_fly_batch_fn(int precision, int dim, bool expl)
{
    return expl ? krylov_batch_fn_form<true>(precision, dim) : krylov_batch_fn_form<false>(precision, dim);
}

size_t krylov_batch_stage_bytes(int precision, int dim)
{
    return krylov_mg_stage_bytes(precision, dim, true);
}

int krylov_fly_batch_blocks(int precision, int dim, size_t smem, bool expl)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void *fn = krylov_fly_batch_fn(precision, dim, expl);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess && fa.maxDynamicSharedSizeBytes < (int)smem)
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, KT, smem);
    if (per > 4) per = 4;
    return sms * per;
}

int launch_krylov_fly_batch(int precision, int dim, const FlyJob *jobs, int njobs, unsigned nblocks,
                            size_t smem, bool expl, cudaStream_t st)
{
    void *args[] = {(void *)&jobs, (void *)&njobs};
    cudaError_t e = cudaLaunchCooperativeKernel(krylov_fly_batch_fn(precision, dim, expl), dim3(nblocks),
                                                dim3(KT), args, smem, st);
    return e == cudaSuccess ? 0 : (int)e;
}

// ---------------------------------------------------------------------------
// a9: corrector and position update (Eqs. VCT_predictor, VCT_update)
// ---------------------------------------------------------------------------
// SUM: the summation pressure gradient of Eq. (gra_sum) (ISPH), rho constant:
// <grad^ p>+_i = sum_j V_j (p_j + p_i) grad w_ij = 2 p_i sum_j V_j grad w_ij +
// sum_j V_j p_ij grad w_ij (both sums kept apart; combined in FP64); else the
// corrected gradient of Eq. (gra_1st).
template <int D, typename R, bool SUM>
__device__ __forceinline__ void corrector_body(const DevParams &P, const Part &c, const Work &W, int n, int bid_)
{
    if (step_failed(W.status)) return;
    int i = bid_ * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (c.type[i] != FLUID) return;
    const int64_t cap = W.cap;
    double xi[3], pi_[3], acci[D];
    load_hat<D>(c, i, xi);
    const float4 hfi = W.hatf[i], lfi = W.hatlo[i];
    load_phys<D>(c, i, pi_);
#pragma unroll
    for (int cc = 0; cc < D; ++cc) acci[cc] = W.acc[(int64_t)cc * cap + i];
    const double p_i = W.pcnt[i] >= 0 ? W.kx[i] : 0.0;
    Acc<R> G[D], Gs[SUM ? D : 1];
    const R inv_l = (R)P.inv_l, ad = (R)P.ad;
    const int cnt = W.nbr_cnt[i];
    for (int k = 0; k < cnt; ++k) {
        int j = W.nbr[(int64_t)k * cap + i];
        int tj = c.type[j];
        if (tj == VIRTUAL) continue;
        R r[D], rr2 = R(0);
        pair_r<D, R>(c, W, j, xi, hfi, lfi, r);
#pragma unroll
        for (int K = 0; K < D; ++K) rr2 += r[K] * r[K];
        if (rr2 == R(0)) continue;
        R rr = sqrt(rr2), w, dw;
        kern_wdw<R>(rr, inv_l, ad, w, dw);
        double pij;
        if (tj == FLUID) {
            pij = (W.pcnt[j] >= 0 ? W.kx[j] : 0.0) - p_i;
        } else {
            double pj[3], s = 0.0;
            load_phys<D>(c, j, pj);
#pragma unroll
            for (int K = 0; K < D; ++K) s += (pj[K] - pi_[K]) * acci[K];
            pij = P.rho * s;
        }
        const R vf = vol_at<R>(W, j) * (-dw / rr);
        R e = vf * (R)pij;
#pragma unroll
        for (int K = 0; K < D; ++K) G[K].add(e * r[K]);
        if constexpr (SUM) {
#pragma unroll
            for (int K = 0; K < D; ++K) Gs[K].add(vf * r[K]);
        }
    }
    double gh[D], g[D];
#pragma unroll
    for (int K = 0; K < D; ++K) {
        double s = 0.0;
        if constexpr (SUM) {
            s = (double)G[K].val() + 2.0 * p_i * (double)Gs[K].val();
        } else {
#pragma unroll
            for (int L2 = 0; L2 < D; ++L2) s += W.L[(int64_t)(K * D + L2) * cap + i] * (double)G[L2].val();
        }
        gh[K] = s;
    }
    jac_apply<D>(c.J[i], c.sx[i], c.sy[i], gh, g);
    double vn[D];
#pragma unroll
    for (int cc = 0; cc < D; ++cc) vn[cc] = W.vstar[(int64_t)cc * cap + i] - P.dt / P.rho * g[cc];
    {
        const int o = c.orig[i];
        W.p_prev2[o] = W.p_prev[o];
        W.p_prev[o] = c.p[i];
        W.p_last[o] = p_i;
    }
    c.p[i] = p_i;
    c.u[i] = vn[0];
    c.x[i] += P.dt * vn[0];
    if (D == 3) {
        c.v[i] = vn[1];
        c.y[i] += P.dt * vn[1];
    }
    c.w[i] = vn[D - 1];
    c.z[i] += P.dt * vn[D - 1];
    bool finite = isfinite(c.x[i]) && isfinite(c.z[i]) && isfinite(p_i) && isfinite(vn[0]) &&
                  isfinite(vn[D - 1]);
    if (!finite) set_error(W.status, VCT_ERR_NONFINITE, i);
}

template <int D, typename R, bool SUM = false>
__global__ void __launch_bounds__(128) k_corrector(DevParams P, Part c, Work W, int n)
{
    corrector_body<D, R, SUM>(P, c, W, n, blockIdx.x);
}

void launch_corrector(const DevParams &P, Part cur, Work W, int64_t n, cudaStream_t st)
{
    unsigned g = (unsigned)((n + 127) / 128);
    if (P.operators == 1) {
        if (P.dim == 2) {
            if (P.precision == VCT_MIXED) k_corrector<2, float, true><<<g, 128, 0, st>>>(P, cur, W, (int)n);
            else k_corrector<2, double, true><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        } else {
            if (P.precision == VCT_MIXED) k_corrector<3, float, true><<<g, 128, 0, st>>>(P, cur, W, (int)n);
            else k_corrector<3, double, true><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        }
        return;
    }
    if (P.dim == 2) {
        if (P.precision == VCT_MIXED) k_corrector<2, float><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        else k_corrector<2, double><<<g, 128, 0, st>>>(P, cur, W, (int)n);
    } else {
        if (P.precision == VCT_MIXED) k_corrector<3, float><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        else k_corrector<3, double><<<g, 128, 0, st>>>(P, cur, W, (int)n);
    }
}

// ---------------------------------------------------------------------------
// Particle regularisation after the position update.  Sec. 4.1 stabilises its
// simulations with optimized particle shifting (shift parameter A), dynamic
// stabilization (allowed overlap of the particle diameter) and XSPH on
// free-surface particles (velocity smoothing eps), and gives only those
// parameters.  The methods, restated from their published forms, act in
// projected space with the step's neighbour lists and the updated positions:
//  * dynamic stabilization: a pair closer than d_DS = (1 - overlap) d0 is
//    pushed apart so that it would be d_DS apart after one step with the
//    corrected velocities, du^_i = -sum mu (d_DS - r)/dt e_ij (mu = 1/2 against
//    a fluid particle, 1 against a wall or virtual one); the velocity gains
//    J^-1 du^ and the position dt J^-1 du^;
//  * XSPH: a free-surface particle takes u_i + eps sum_{j fluid} V0 (u_j - u_i) w_ij;
//  * shifting: dr^_i = -A l |v^_i| dt grad^C_i, grad^C_i = sum_j V0 grad w_ij
//    over all neighbours, v^ = J v; a free-surface particle keeps only the part
//    tangential to the surface, whose normal is -L grad^C normalised with
//    L = B^-1, B = sum_j V0 (r^_j - r^_i) (x) grad w_ij (none if B is singular).
// Projected displacements return through the Jacobian at the new position
// (dz = (dz^ - s_x dx^ - s_y dy^)/alpha).  Pair sums run in list order, in FP64
// (FP64 form) or compensated FP32 on FP64 differences (mixed form); the
// corrections themselves are FP64.  A particle's correction reads only copies
// made before the kernel writes, so the result does not depend on the thread
// order.
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void reg_to_phys(double J, double sx, double sy, const double *dh, double *dp)
{
    dp[0] = dh[0];
    if (D == 2) {
        dp[1] = (dh[1] - sx * dh[0]) / J;
    } else {
        dp[1] = dh[1];
        dp[2] = (dh[2] - sx * dh[0] - sy * dh[1]) / J;
    }
}

// In-place inverse of a D x D matrix by Gaussian elimination with partial
// pivoting; false when a pivot falls below 1e-14 of the largest entry.
template <int D>
__device__ bool reg_invert(double (&A)[D * D], double (&X)[D * D])
{
    double amax = 0.0;
#pragma unroll
    for (int q = 0; q < D * D; ++q) amax = fmax(amax, fabs(A[q]));
    if (!(amax > 0.0)) return false;
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int c = 0; c < D; ++c) X[r * D + c] = r == c ? 1.0 : 0.0;
    for (int k = 0; k < D; ++k) {
        int piv = k;
        for (int r = k + 1; r < D; ++r)
            if (fabs(A[r * D + k]) > fabs(A[piv * D + k])) piv = r;
        if (!(fabs(A[piv * D + k]) > 1e-14 * amax)) return false;
        if (piv != k)
            for (int c = 0; c < D; ++c) {
                double t = A[k * D + c]; A[k * D + c] = A[piv * D + c]; A[piv * D + c] = t;
                t = X[k * D + c]; X[k * D + c] = X[piv * D + c]; X[piv * D + c] = t;
            }
        for (int r = k + 1; r < D; ++r) {
            const double f = A[r * D + k] / A[k * D + k];
            for (int c = k; c < D; ++c) A[r * D + c] -= f * A[k * D + c];
            for (int c = 0; c < D; ++c) X[r * D + c] -= f * X[k * D + c];
        }
    }
    for (int k = D - 1; k >= 0; --k)
        for (int c = 0; c < D; ++c) {
            double s = X[k * D + c];
            for (int j = k + 1; j < D; ++j) s -= A[k * D + j] * X[j * D + c];
            X[k * D + c] = s / A[k * D + k];
        }
    return true;
}

// Projected positions and metric at the updated positions; velocity copies.
template <int D>
__device__ __forceinline__ void reg_geom_body(const DevParams &P, const Part &c, const Work &W, int n, int bid_)
{
    if (step_failed(W.status)) return;
    const int i = bid_ * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t cap = W.cap;
    double zh, J, sx, sy, c0, c3;
    const double y = D == 3 ? c.y[i] : 0.0;
    map_metric(P, c.x[i], y, c.z[i], zh, J, sx, sy, c0, c3);
    W.rxh[i] = c.x[i];
    if (D == 3) W.rxh[cap + i] = y;
    W.rxh[(D - 1) * cap + i] = zh;
    {   // hi/lo FP32 copy for the mixed form's pair differences (the step's copy
        // is no longer needed: the next step's reorder writes it again)
        float4 lo;
        W.hatf[i] = f4_hilo_split(c.x[i], y, zh, lo);
        W.hatlo[i] = lo;
    }
    W.rmet[i] = J;
    W.rmet[cap + i] = sx;
    W.rmet[2 * cap + i] = sy;
    W.rud[i] = c.u[i];
    if (D == 3) W.rud[cap + i] = c.v[i];
    W.rud[(D - 1) * cap + i] = c.w[i];
#pragma unroll
    for (int K = 0; K < D; ++K) W.rdh[K * cap + i] = 0.0;
}

template <int D>
__global__ void __launch_bounds__(128) k_reg_geom(DevParams P, Part c, Work W, int n)
{
    reg_geom_body<D>(P, c, W, n, blockIdx.x);
}

template <int D>
__device__ __forceinline__ void reg_load(const Work &W, int i, double *x)
{
#pragma unroll
    for (int K = 0; K < D; ++K) x[K] = W.rxh[K * W.cap + i];
}

// Dynamic stabilization: corrected velocity copy and projected displacement.
// R: precision of the pair terms (FP64 form: double; mixed form: float, the
// differences formed in FP64 first).
template <int D, typename R>
__device__ __forceinline__ void reg_ds_body(const DevParams &P, const Part &c, const Work &W, int n, int bid_)
{
    if (step_failed(W.status)) return;
    const int i = bid_ * blockDim.x + threadIdx.x;
    if (i >= n || c.type[i] != FLUID) return;
    const int64_t cap = W.cap;
    const double dds = (1.0 - P.ds_overlap) * P.d0;
    const R ddsr = (R)dds, dtr = (R)P.dt;
    double xi[D];
    R du[D];
    reg_load<D>(W, i, xi);
    const float4 hfi = W.hatf[i], lfi = W.hatlo[i];
#pragma unroll
    for (int K = 0; K < D; ++K) du[K] = R(0);
    const int cnt = W.nbr_cnt[i];
    for (int k = 0; k < cnt; ++k) {
        const int j = W.nbr[(int64_t)k * cap + i];
        R r[D], r2 = R(0);
        if constexpr (sizeof(R) == sizeof(float)) {   // mixed: hi/lo differences
            hilo_diff<D>(W.hatf[j], W.hatlo[j], hfi, lfi, r);
        } else {
            double xj[D];
            reg_load<D>(W, j, xj);
#pragma unroll
            for (int K = 0; K < D; ++K) r[K] = (R)(xj[K] - xi[K]);
        }
#pragma unroll
        for (int K = 0; K < D; ++K) r2 += r[K] * r[K];
        const R rr = sqrt(r2);
        if (!(rr < ddsr) || rr == R(0)) continue;
        const R f = (c.type[j] == FLUID ? R(0.5) : R(1)) * (ddsr - rr) / (dtr * rr);
#pragma unroll
        for (int K = 0; K < D; ++K) du[K] -= f * r[K];
    }
    double dud[D], dv[D];
#pragma unroll
    for (int K = 0; K < D; ++K) dud[K] = (double)du[K];
    reg_to_phys<D>(W.rmet[i], W.rmet[cap + i], W.rmet[2 * cap + i], dud, dv);
#pragma unroll
    for (int K = 0; K < D; ++K) {
        W.rud[K * cap + i] += dv[K];
        W.rdh[K * cap + i] = P.dt * dud[K];
    }
}

template <int D, typename R>
__global__ void __launch_bounds__(128) k_reg_ds(DevParams P, Part c, Work W, int n)
{
    reg_ds_body<D, R>(P, c, W, n, blockIdx.x);
}

// XSPH on free-surface particles, shifting, and the final write of the state.
template <int D, typename R>
__device__ __forceinline__ void reg_apply_body(const DevParams &P, const Part &c, const Work &W, int n, int bid_)
{
    if (step_failed(W.status)) return;
    const int i = bid_ * blockDim.x + threadIdx.x;
    if (i >= n || c.type[i] != FLUID) return;
    const int64_t cap = W.cap;
    const R inv_l = (R)P.inv_l, ad = (R)P.ad, V0 = (R)P.V0;
    const bool fsi = W.fs[i] != 0;
    const bool do_x = P.xsph_eps > 0.0 && fsi, do_s = P.ops_shift > 0.0;
    double xi[D], ui[D], gc[D], xs[D], B[D * D];
    Acc<R> gca[D], xsa[D], Ba[D * D];
    reg_load<D>(W, i, xi);
#pragma unroll
    for (int K = 0; K < D; ++K) ui[K] = W.rud[K * cap + i];
    const int cnt = (do_x || do_s) ? W.nbr_cnt[i] : 0;
    const float4 hfi = W.hatf[i], lfi = W.hatlo[i];
    for (int k = 0; k < cnt; ++k) {
        const int j = W.nbr[(int64_t)k * cap + i];
        R r[D], r2 = R(0);
        if constexpr (sizeof(R) == sizeof(float)) {   // mixed: hi/lo differences, r = x_i - x_j
            hilo_diff<D>(hfi, lfi, W.hatf[j], W.hatlo[j], r);
        } else {
            double xj[D];
            reg_load<D>(W, j, xj);
#pragma unroll
            for (int K = 0; K < D; ++K) r[K] = (R)(xi[K] - xj[K]);
        }
#pragma unroll
        for (int K = 0; K < D; ++K) r2 += r[K] * r[K];
        const R rr = sqrt(r2);
        if (rr == R(0)) continue;
        R w, dw;
        kern_wdw<R>(rr, inv_l, ad, w, dw);
        if (do_x && c.type[j] == FLUID) {
#pragma unroll
            for (int K = 0; K < D; ++K) xsa[K].add(V0 * (R)(W.rud[K * cap + j] - ui[K]) * w);
        }
        if (do_s) {
            const R dwr = dw / rr;
#pragma unroll
            for (int K = 0; K < D; ++K) gca[K].add(V0 * dwr * r[K]);
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
                for (int b = 0; b < D; ++b) Ba[a * D + b].add(-(V0 * dwr * r[a] * r[b]));
        }
    }
#pragma unroll
    for (int K = 0; K < D; ++K) {
        gc[K] = (double)gca[K].val();
        xs[K] = (double)xsa[K].val();
    }
#pragma unroll
    for (int q = 0; q < D * D; ++q) B[q] = (double)Ba[q].val();
    double un[D], dh[D];
#pragma unroll
    for (int K = 0; K < D; ++K) {
        un[K] = do_x ? ui[K] + P.xsph_eps * xs[K] : ui[K];
        dh[K] = W.rdh[K * cap + i];
    }
    if (do_s) {
        const double J = W.rmet[i], sx = W.rmet[cap + i], sy = W.rmet[2 * cap + i];
        double vh[D];
        vh[0] = un[0];
        if (D == 2) {
            vh[1] = sx * un[0] + J * un[1];
        } else {
            vh[1] = un[1];
            vh[2] = sx * un[0] + sy * un[1] + J * un[2];
        }
        double sp = 0.0;
#pragma unroll
        for (int K = 0; K < D; ++K) sp += vh[K] * vh[K];
        const double Df = P.ops_shift * P.l * sqrt(sp) * P.dt;
        double s[D];
#pragma unroll
        for (int K = 0; K < D; ++K) s[K] = -Df * gc[K];
        if (fsi) {
            double Li[D * D], nv[D], nn = 0.0;
            const bool ok = reg_invert<D>(B, Li);
            if (ok) {
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    nv[a] = 0.0;
#pragma unroll
                    for (int b = 0; b < D; ++b) nv[a] -= Li[a * D + b] * gc[b];
                    nn += nv[a] * nv[a];
                }
            }
            if (!ok || !(nn > 0.0)) {
#pragma unroll
                for (int K = 0; K < D; ++K) s[K] = 0.0;
            } else {
                nn = sqrt(nn);
                double sn = 0.0;
#pragma unroll
                for (int K = 0; K < D; ++K) {
                    nv[K] /= nn;
                    sn += s[K] * nv[K];
                }
#pragma unroll
                for (int K = 0; K < D; ++K) s[K] -= sn * nv[K];
            }
        }
#pragma unroll
        for (int K = 0; K < D; ++K) dh[K] += s[K];
    }
    double dp[D];
    reg_to_phys<D>(W.rmet[i], W.rmet[cap + i], W.rmet[2 * cap + i], dh, dp);
    c.x[i] += dp[0];
    c.u[i] = un[0];
    if (D == 3) {
        c.y[i] += dp[1];
        c.v[i] = un[1];
    }
    c.z[i] += dp[D - 1];
    c.w[i] = un[D - 1];
    if (!(isfinite(c.x[i]) && isfinite(c.z[i]) && isfinite(un[0]) && isfinite(un[D - 1])))
        set_error(W.status, VCT_ERR_NONFINITE, i);
}

template <int D, typename R>
__global__ void __launch_bounds__(128) k_reg_apply(DevParams P, Part c, Work W, int n)
{
    reg_apply_body<D, R>(P, c, W, n, blockIdx.x);
}

bool regularise_on(const DevParams &P)
{
    return P.ops_shift > 0.0 || P.ds_overlap > 0.0 || P.xsph_eps > 0.0;
}

int launch_regularise(const DevParams &P, Part cur, Work W, int64_t n, cudaStream_t st)
{
    if (!regularise_on(P)) return 0;
    const unsigned g = (unsigned)((n + 127) / 128);
    const bool mixed = P.precision == VCT_MIXED;
    if (P.dim == 2) {
        k_reg_geom<2><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        if (P.ds_overlap > 0.0) {
            if (mixed) k_reg_ds<2, float><<<g, 128, 0, st>>>(P, cur, W, (int)n);
            else k_reg_ds<2, double><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        }
        if (mixed) k_reg_apply<2, float><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        else k_reg_apply<2, double><<<g, 128, 0, st>>>(P, cur, W, (int)n);
    } else {
        k_reg_geom<3><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        if (P.ds_overlap > 0.0) {
            if (mixed) k_reg_ds<3, float><<<g, 128, 0, st>>>(P, cur, W, (int)n);
            else k_reg_ds<3, double><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        }
        if (mixed) k_reg_apply<3, float><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        else k_reg_apply<3, double><<<g, 128, 0, st>>>(P, cur, W, (int)n);
    }
    return P.ds_overlap > 0.0 ? 3 : 2;
}

// ---------------------------------------------------------------------------
// sph2_derivatives: corrected gradient + SPH(2) of caller fields
// ---------------------------------------------------------------------------
template <int D, typename R>
__global__ void __launch_bounds__(128) k_sph2_field(DevParams P, const Part c, Work W, int n,
                                                    const double *phi, int ncomp,
                                                    double *grad, double *d2, double *lap)
{
    constexpr int M = D == 2 ? 3 : 6;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int o = c.orig[i];
    if (c.type[i] != FLUID) {
        for (int cc = 0; cc < ncomp; ++cc) {
            if (grad) for (int K = 0; K < D; ++K) grad[((int64_t)cc * D + K) * n + o] = 0.0;
            if (d2) for (int a = 0; a < M; ++a) d2[((int64_t)cc * M + a) * n + o] = 0.0;
            if (lap) lap[(int64_t)cc * n + o] = 0.0;
        }
        return;
    }
    const int64_t cap = W.cap;
    double xi[3];
    load_hat<D>(c, i, xi);
    R L[D * D], Ct[D * M];
#pragma unroll
    for (int k = 0; k < D * D; ++k) L[k] = (R)W.L[(int64_t)k * cap + i];
#pragma unroll
    for (int k = 0; k < D * M; ++k) Ct[k] = (R)W.Ct[(int64_t)k * cap + i];
    const R inv_l = (R)P.inv_l, ad = (R)P.ad;
    const int cnt = W.nbr_cnt[i];
    Acc<R> Mm[M * M];
    for (int k = 0; k < cnt; ++k) {
        int j = W.nbr[(int64_t)k * cap + i];
        if (c.type[j] == VIRTUAL) continue;
        double xj[3];
        load_hat<D>(c, j, xj);
        R r[D], rr2 = R(0);
#pragma unroll
        for (int K = 0; K < D; ++K) {
            r[K] = (R)(xj[K] - xi[K]);
            rr2 += r[K] * r[K];
        }
        if (rr2 == R(0)) continue;
        R rr = sqrt(rr2), w, dw;
        kern_wdw<R>(rr, inv_l, ad, w, dw);
        R gw[D], fac = -dw / rr, rg = R(0);
#pragma unroll
        for (int K = 0; K < D; ++K) gw[K] = fac * r[K];
#pragma unroll
        for (int K = 0; K < D; ++K) {
            R s = R(0);
#pragma unroll
            for (int L2 = 0; L2 < D; ++L2) s += L[K * D + L2] * gw[L2];
            rg += r[K] * s;
        }
        R VF = (R)vol_of(P, c, j) * rg / (rr2 * rr2), q[M], pv[M];
        qvec<D, R>(r, q);
#pragma unroll
        for (int a = 0; a < M; ++a) {
            R s = R(0);
#pragma unroll
            for (int K = 0; K < D; ++K) s += Ct[K * M + a] * r[K];
            pv[a] = q[a] - s;
        }
#pragma unroll
        for (int a = 0; a < M; ++a)
#pragma unroll
            for (int b = 0; b < M; ++b) Mm[a * M + b].add(VF * q[a] * pv[b]);
    }
    double ct[M];
    ctilde<D>(c.c3[i], c.sx[i], c.sy[i], ct);
    for (int cc = 0; cc < ncomp; ++cc) {
        const double *f = phi + (int64_t)cc * n;
        const double fi = f[o];
        Acc<R> G[D];
        for (int k = 0; k < cnt; ++k) {
            int j = W.nbr[(int64_t)k * cap + i];
            if (c.type[j] == VIRTUAL) continue;
            double xj[3];
            load_hat<D>(c, j, xj);
            R r[D], rr2 = R(0);
#pragma unroll
            for (int K = 0; K < D; ++K) {
                r[K] = (R)(xj[K] - xi[K]);
                rr2 += r[K] * r[K];
            }
            if (rr2 == R(0)) continue;
            R rr = sqrt(rr2), w, dw;
            kern_wdw<R>(rr, inv_l, ad, w, dw);
            R e = (R)vol_of(P, c, j) * (R)(f[c.orig[j]] - fi) * (-dw / rr);
#pragma unroll
            for (int K = 0; K < D; ++K) G[K].add(e * r[K]);
        }
        double g[D];
#pragma unroll
        for (int K = 0; K < D; ++K) {
            double s = 0.0;
#pragma unroll
            for (int L2 = 0; L2 < D; ++L2) s += W.L[(int64_t)(K * D + L2) * cap + i] * (double)G[L2].val();
            g[K] = s;
        }
        Acc<R> b[M];
        for (int k = 0; k < cnt; ++k) {
            int j = W.nbr[(int64_t)k * cap + i];
            if (c.type[j] == VIRTUAL) continue;
            double xj[3];
            load_hat<D>(c, j, xj);
            R r[D], rr2 = R(0);
            double rgd = 0.0;
#pragma unroll
            for (int K = 0; K < D; ++K) {
                double rdk = xj[K] - xi[K];
                r[K] = (R)rdk;
                rr2 += r[K] * r[K];
                rgd += rdk * g[K];
            }
            if (rr2 == R(0)) continue;
            R rr = sqrt(rr2), w, dw;
            kern_wdw<R>(rr, inv_l, ad, w, dw);
            R gw[D], fac = -dw / rr, rg = R(0);
#pragma unroll
            for (int K = 0; K < D; ++K) gw[K] = fac * r[K];
#pragma unroll
            for (int K = 0; K < D; ++K) {
                R s = R(0);
#pragma unroll
                for (int L2 = 0; L2 < D; ++L2) s += L[K * D + L2] * gw[L2];
                rg += r[K] * s;
            }
            if (P.operators == 1) {   // ISPH: D_a = sum_j V_j k_a(r_ij) phi_ij (Eq. sec_0th)
                R kw[M];
                er_weights<D, R>(r, rr2, fac, kw);
                R e0 = (R)vol_of(P, c, j) * (R)(f[c.orig[j]] - fi);
#pragma unroll
                for (int a = 0; a < M; ++a) b[a].add(e0 * kw[a]);
                continue;
            }
            R VF = (R)vol_of(P, c, j) * rg / (rr2 * rr2), q[M];
            qvec<D, R>(r, q);
            // phi_ij - r_ij . <grad phi>_i formed in FP64 (cancellation), summed in R
            R e = VF * (R)((f[c.orig[j]] - fi) - rgd);
#pragma unroll
            for (int a = 0; a < M; ++a) b[a].add(e * q[a]);
        }
        double A[M * M], bb[M];
#pragma unroll
        for (int k = 0; k < M * M; ++k) A[k] = (double)Mm[k].val();
#pragma unroll
        for (int a = 0; a < M; ++a) bb[a] = (double)b[a].val();
        if (W.fs[i] == 2) {   // isolated particle: no derivatives
#pragma unroll
            for (int a = 0; a < M; ++a) bb[a] = 0.0;
        } else if (P.operators != 1) {
            if (!lu_solve<M, 1>(A, bb)) {
                if (!W.fs[i]) set_error(W.status, VCT_ERR_SINGULAR, i);
#pragma unroll
                for (int a = 0; a < M; ++a) bb[a] = 0.0;
            }
#pragma unroll
            for (int a = 0; a < M; ++a) bb[a] *= 2.0;   // D = 2 M^-1 b
        }
        if (grad)
            for (int K = 0; K < D; ++K) grad[((int64_t)cc * D + K) * n + o] = g[K];
        if (d2)
            for (int a = 0; a < M; ++a) d2[((int64_t)cc * M + a) * n + o] = a < D ? bb[a] : 0.5 * bb[a];
        if (lap) {
            double s = c.c0[i] * g[D - 1];
#pragma unroll
            for (int a = 0; a < M; ++a) s += ct[a] * bb[a];
            lap[(int64_t)cc * n + o] = s;
        }
    }
}

void launch_sph2_field(const DevParams &P, Part cur, Work W, int64_t n, const double *phi,
                       int ncomp, double *grad, double *d2, double *lap, cudaStream_t st)
{
    unsigned g = (unsigned)((n + 127) / 128);
    if (P.dim == 2) {
        if (P.precision == VCT_MIXED)
            k_sph2_field<2, float><<<g, 128, 0, st>>>(P, cur, W, (int)n, phi, ncomp, grad, d2, lap);
        else k_sph2_field<2, double><<<g, 128, 0, st>>>(P, cur, W, (int)n, phi, ncomp, grad, d2, lap);
    } else {
        if (P.precision == VCT_MIXED)
            k_sph2_field<3, float><<<g, 128, 0, st>>>(P, cur, W, (int)n, phi, ncomp, grad, d2, lap);
        else k_sph2_field<3, double><<<g, 128, 0, st>>>(P, cur, W, (int)n, phi, ncomp, grad, d2, lap);
    }
}

// ---------------------------------------------------------------------------
// a12 (operator part): adjoint of sph2_derivatives with respect to the field.
// For fluid particle i the outputs are linear in phi_ij = phi_j - phi_i:
//   g_i = L_i sum_j V_j phi_ij grad w_ij,
//   D_i = 2 M_i^-1 sum_j V_j F_ij q_ij (phi_ij - r_ij . g_i)      (Eq. sec_SPH2)
//   d2_i = H D_i (cross entries halved),  lap_i = c0 g_i,z + c~ . D_i (Eq. lap_VCT)
// Given the output adjoints, pass 1 forms per particle
//   Dbar = H d2bar + c~ lapbar,  bbar = 2 M_i^-T Dbar   (adjoint of the small solve)
//   gbar' = gbar + c0 lapbar e_z - sum_j V_j F_ij (bbar . q_ij) r_ij,
// and each pair (i, j) carries w_ij = V_j [F_ij (bbar_i . q_ij) + (L_i grad w_ij) . gbar'_i];
// pass 2 gathers phibar_j = sum_{i : j in S_i} w_ij - sum_{k in S_j} w_jk over the
// symmetric neighbour relation (the transpose scatter written as a gather).
// ---------------------------------------------------------------------------
template <int D, typename R>
__global__ void __launch_bounds__(128) k_sph2_adj1(DevParams P, const Part c, Work W, int n,
                                                   const double *gbar, const double *d2bar,
                                                   const double *lapbar, int comp)
{
    constexpr int M = D == 2 ? 3 : 6;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t cap = W.cap;
    if (c.type[i] != FLUID) {
        for (int a = 0; a < M + D; ++a) W.adj[(int64_t)a * cap + i] = 0.0;
        return;
    }
    const int o = c.orig[i];
    double xi[3];
    load_hat<D>(c, i, xi);
    R L[D * D], Ct[D * M];
#pragma unroll
    for (int k = 0; k < D * D; ++k) L[k] = (R)W.L[(int64_t)k * cap + i];
#pragma unroll
    for (int k = 0; k < D * M; ++k) Ct[k] = (R)W.Ct[(int64_t)k * cap + i];
    const R inv_l = (R)P.inv_l, ad = (R)P.ad;
    const int cnt = W.nbr_cnt[i];
    Acc<R> Mm[M * M];
    for (int k = 0; k < cnt; ++k) {
        int j = W.nbr[(int64_t)k * cap + i];
        if (c.type[j] == VIRTUAL) continue;
        double xj[3];
        load_hat<D>(c, j, xj);
        R r[D], rr2 = R(0);
#pragma unroll
        for (int K = 0; K < D; ++K) {
            r[K] = (R)(xj[K] - xi[K]);
            rr2 += r[K] * r[K];
        }
        if (rr2 == R(0)) continue;
        R rr = sqrt(rr2), w, dw;
        kern_wdw<R>(rr, inv_l, ad, w, dw);
        R gw[D], fac = -dw / rr, rg = R(0);
#pragma unroll
        for (int K = 0; K < D; ++K) gw[K] = fac * r[K];
#pragma unroll
        for (int K = 0; K < D; ++K) {
            R s = R(0);
#pragma unroll
            for (int L2 = 0; L2 < D; ++L2) s += L[K * D + L2] * gw[L2];
            rg += r[K] * s;
        }
        R VF = (R)vol_of(P, c, j) * rg / (rr2 * rr2), q[M], pv[M];
        qvec<D, R>(r, q);
#pragma unroll
        for (int a = 0; a < M; ++a) {
            R s = R(0);
#pragma unroll
            for (int K = 0; K < D; ++K) s += Ct[K * M + a] * r[K];
            pv[a] = q[a] - s;
        }
#pragma unroll
        for (int a = 0; a < M; ++a)
#pragma unroll
            for (int b = 0; b < M; ++b) Mm[a * M + b].add(VF * q[a] * pv[b]);
    }
    double ct[M];
    ctilde<D>(c.c3[i], c.sx[i], c.sy[i], ct);
    const double lb = lapbar ? lapbar[(int64_t)comp * n + o] : 0.0;
    double Dbar[M], gb[D];
#pragma unroll
    for (int a = 0; a < M; ++a) {
        const double d2b = d2bar ? d2bar[((int64_t)comp * M + a) * n + o] : 0.0;
        Dbar[a] = (a < D ? d2b : 0.5 * d2b) + ct[a] * lb;
    }
#pragma unroll
    for (int K = 0; K < D; ++K) gb[K] = gbar ? gbar[((int64_t)comp * D + K) * n + o] : 0.0;
    gb[D - 1] += c.c0[i] * lb;
    // bbar = 2 M^-T Dbar
    double A[M * M];
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int b = 0; b < M; ++b) A[a * M + b] = (double)Mm[b * M + a].val();
    // as in the forward operator: an isolated particle has no second derivatives,
    // and a free-surface particle whose M_i cannot be factored loses them
    const int fsi = W.fs[i];
    if (fsi == 2 || !lu_solve<M, 1>(A, Dbar)) {
        if (!fsi) set_error(W.status, VCT_ERR_SINGULAR, i);
#pragma unroll
        for (int a = 0; a < M; ++a) Dbar[a] = 0.0;
    }
    R bb[M];
#pragma unroll
    for (int a = 0; a < M; ++a) bb[a] = (R)(2.0 * Dbar[a]);
    // gbar' = gbar - sum_j V F (bbar . q) r
    Acc<R> u[D];
    for (int k = 0; k < cnt; ++k) {
        int j = W.nbr[(int64_t)k * cap + i];
        if (c.type[j] == VIRTUAL) continue;
        double xj[3];
        load_hat<D>(c, j, xj);
        R r[D], rr2 = R(0);
#pragma unroll
        for (int K = 0; K < D; ++K) {
            r[K] = (R)(xj[K] - xi[K]);
            rr2 += r[K] * r[K];
        }
        if (rr2 == R(0)) continue;
        R rr = sqrt(rr2), w, dw;
        kern_wdw<R>(rr, inv_l, ad, w, dw);
        R fac = -dw / rr, rg = R(0);
#pragma unroll
        for (int K = 0; K < D; ++K) {
            R s = R(0);
#pragma unroll
            for (int L2 = 0; L2 < D; ++L2) s += L[K * D + L2] * fac * r[L2];
            rg += r[K] * s;
        }
        R VF = (R)vol_of(P, c, j) * rg / (rr2 * rr2), q[M], bq = R(0);
        qvec<D, R>(r, q);
#pragma unroll
        for (int a = 0; a < M; ++a) bq += bb[a] * q[a];
#pragma unroll
        for (int K = 0; K < D; ++K) u[K].add(VF * bq * r[K]);
    }
#pragma unroll
    for (int a = 0; a < M; ++a) W.adj[(int64_t)a * cap + i] = (double)bb[a];
#pragma unroll
    for (int K = 0; K < D; ++K) W.adj[(int64_t)(M + K) * cap + i] = gb[K] - (double)u[K].val();
}

// Pair weight w_ij seen from particle i (the owner of the outputs) for neighbour j.
template <int D, typename R>
__device__ __forceinline__ R adj_pair(const DevParams &P, const Part &c, const Work &W, int i, int j,
                                      const double *xi, const double *xj)
{
    constexpr int M = D == 2 ? 3 : 6;
    const int64_t cap = W.cap;
    R r[D], rr2 = R(0);
#pragma unroll
    for (int K = 0; K < D; ++K) {
        r[K] = (R)(xj[K] - xi[K]);
        rr2 += r[K] * r[K];
    }
    if (rr2 == R(0)) return R(0);
    R rr = sqrt(rr2), w, dw;
    kern_wdw<R>(rr, (R)P.inv_l, (R)P.ad, w, dw);
    R fac = -dw / rr, gt[D], rg = R(0);
#pragma unroll
    for (int K = 0; K < D; ++K) {
        R s = R(0);
#pragma unroll
        for (int L2 = 0; L2 < D; ++L2) s += (R)W.L[(int64_t)(K * D + L2) * cap + i] * fac * r[L2];
        gt[K] = s;
        rg += r[K] * s;
    }
    R F = rg / (rr2 * rr2), q[M], bq = R(0), gg = R(0);
    qvec<D, R>(r, q);
#pragma unroll
    for (int a = 0; a < M; ++a) bq += (R)W.adj[(int64_t)a * cap + i] * q[a];
#pragma unroll
    for (int K = 0; K < D; ++K) gg += gt[K] * (R)W.adj[(int64_t)(M + K) * cap + i];
    return (R)vol_of(P, c, j) * (F * bq + gg);
}

template <int D, typename R>
__global__ void __launch_bounds__(128) k_sph2_adj2(DevParams P, const Part c, Work W, int n,
                                                   double *phibar, int comp)
{
    int jdx = blockIdx.x * blockDim.x + threadIdx.x;
    if (jdx >= n) return;
    const int o = c.orig[jdx];
    const int tj = c.type[jdx];
    if (tj == VIRTUAL) {
        phibar[(int64_t)comp * n + o] = 0.0;
        return;
    }
    const int64_t cap = W.cap;
    double xj[3];
    load_hat<D>(c, jdx, xj);
    Acc<R> acc;
    const int cnt = W.nbr_cnt[jdx];
    for (int k = 0; k < cnt; ++k) {
        const int i = W.nbr[(int64_t)k * cap + jdx];
        const int ti = c.type[i];
        if (ti == VIRTUAL) continue;
        double xi[3];
        load_hat<D>(c, i, xi);
        if (ti == FLUID) acc.add(adj_pair<D, R>(P, c, W, i, jdx, xi, xj));        // incoming w_ij
        if (tj == FLUID) acc.add(-adj_pair<D, R>(P, c, W, jdx, i, xj, xi));       // outgoing w_ji
    }
    phibar[(int64_t)comp * n + o] = (double)acc.val();
}

// The same adjoint for NC <= 3 fields at once: M_i is summed and factored once
// and solved for the NC right sides, each pair's geometry is formed once for all
// fields (the forward operator shares them the same way).  W.adj holds the NC
// fields' (bbar, gbar') rows one after the other.
template <int D, typename R, int NC>
__global__ void __launch_bounds__(128) k_sph2_adjm1(DevParams P, const Part c, Work W, int n,
                                                    const double *gbar, const double *d2bar,
                                                    const double *lapbar)
{
    constexpr int M = D == 2 ? 3 : 6, S = M + D;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t cap = W.cap;
    if (c.type[i] != FLUID) {
        for (int a = 0; a < NC * S; ++a) W.adj[(int64_t)a * cap + i] = 0.0;
        return;
    }
    const int o = c.orig[i];
    double xi[3];
    load_hat<D>(c, i, xi);
    R L[D * D], Ct[D * M];
#pragma unroll
    for (int k = 0; k < D * D; ++k) L[k] = (R)W.L[(int64_t)k * cap + i];
#pragma unroll
    for (int k = 0; k < D * M; ++k) Ct[k] = (R)W.Ct[(int64_t)k * cap + i];
    const R inv_l = (R)P.inv_l, ad = (R)P.ad;
    const int cnt = W.nbr_cnt[i];
    Acc<R> Mm[M * M];
    for (int k = 0; k < cnt; ++k) {
        int j = W.nbr[(int64_t)k * cap + i];
        if (c.type[j] == VIRTUAL) continue;
        double xj[3];
        load_hat<D>(c, j, xj);
        R r[D], rr2 = R(0);
#pragma unroll
        for (int K = 0; K < D; ++K) {
            r[K] = (R)(xj[K] - xi[K]);
            rr2 += r[K] * r[K];
        }
        if (rr2 == R(0)) continue;
        R rr = sqrt(rr2), w, dw;
        kern_wdw<R>(rr, inv_l, ad, w, dw);
        R gw[D], fac = -dw / rr, rg = R(0);
#pragma unroll
        for (int K = 0; K < D; ++K) gw[K] = fac * r[K];
#pragma unroll
        for (int K = 0; K < D; ++K) {
            R s2 = R(0);
#pragma unroll
            for (int L2 = 0; L2 < D; ++L2) s2 += L[K * D + L2] * gw[L2];
            rg += r[K] * s2;
        }
        R VF = (R)vol_of(P, c, j) * rg / (rr2 * rr2), q[M], pv[M];
        qvec<D, R>(r, q);
#pragma unroll
        for (int a = 0; a < M; ++a) {
            R s2 = R(0);
#pragma unroll
            for (int K = 0; K < D; ++K) s2 += Ct[K * M + a] * r[K];
            pv[a] = q[a] - s2;
        }
#pragma unroll
        for (int a = 0; a < M; ++a)
#pragma unroll
            for (int b = 0; b < M; ++b) Mm[a * M + b].add(VF * q[a] * pv[b]);
    }
    double ct[M];
    ctilde<D>(c.c3[i], c.sx[i], c.sy[i], ct);
    double Dbar[M * NC], gb[NC][D];   // Dbar row-major M x NC
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) {
        const double lb = lapbar ? lapbar[(int64_t)cc * n + o] : 0.0;
#pragma unroll
        for (int a = 0; a < M; ++a) {
            const double d2b = d2bar ? d2bar[((int64_t)cc * M + a) * n + o] : 0.0;
            Dbar[a * NC + cc] = (a < D ? d2b : 0.5 * d2b) + ct[a] * lb;
        }
#pragma unroll
        for (int K = 0; K < D; ++K) gb[cc][K] = gbar ? gbar[((int64_t)cc * D + K) * n + o] : 0.0;
        gb[cc][D - 1] += c.c0[i] * lb;
    }
    double A[M * M];
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
        for (int b = 0; b < M; ++b) A[a * M + b] = (double)Mm[b * M + a].val();
    const int fsi = W.fs[i];
    if (fsi == 2 || !lu_solve<M, NC>(A, Dbar)) {
        if (!fsi) set_error(W.status, VCT_ERR_SINGULAR, i);
#pragma unroll
        for (int a = 0; a < M * NC; ++a) Dbar[a] = 0.0;
    }
    R bb[NC][M];
#pragma unroll
    for (int cc = 0; cc < NC; ++cc)
#pragma unroll
        for (int a = 0; a < M; ++a) bb[cc][a] = (R)(2.0 * Dbar[a * NC + cc]);
    Acc<R> u[NC][D];
    for (int k = 0; k < cnt; ++k) {
        int j = W.nbr[(int64_t)k * cap + i];
        if (c.type[j] == VIRTUAL) continue;
        double xj[3];
        load_hat<D>(c, j, xj);
        R r[D], rr2 = R(0);
#pragma unroll
        for (int K = 0; K < D; ++K) {
            r[K] = (R)(xj[K] - xi[K]);
            rr2 += r[K] * r[K];
        }
        if (rr2 == R(0)) continue;
        R rr = sqrt(rr2), w, dw;
        kern_wdw<R>(rr, inv_l, ad, w, dw);
        R fac = -dw / rr, rg = R(0);
#pragma unroll
        for (int K = 0; K < D; ++K) {
            R s2 = R(0);
#pragma unroll
            for (int L2 = 0; L2 < D; ++L2) s2 += L[K * D + L2] * fac * r[L2];
            rg += r[K] * s2;
        }
        R VF = (R)vol_of(P, c, j) * rg / (rr2 * rr2), q[M];
        qvec<D, R>(r, q);
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) {
            R bq = R(0);
#pragma unroll
            for (int a = 0; a < M; ++a) bq += bb[cc][a] * q[a];
#pragma unroll
            for (int K = 0; K < D; ++K) u[cc][K].add(VF * bq * r[K]);
        }
    }
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) {
#pragma unroll
        for (int a = 0; a < M; ++a) W.adj[(int64_t)(cc * S + a) * cap + i] = (double)bb[cc][a];
#pragma unroll
        for (int K = 0; K < D; ++K)
            W.adj[(int64_t)(cc * S + M + K) * cap + i] = gb[cc][K] - (double)u[cc][K].val();
    }
}

// Pair weights w_ij of the NC fields seen from particle i (the owner) for neighbour j.
template <int D, typename R, int NC>
__device__ __forceinline__ void adj_pair_m(const DevParams &P, const Part &c, const Work &W, int i,
                                           int j, const double *xi, const double *xj, R *wout)
{
    constexpr int M = D == 2 ? 3 : 6, S = M + D;
    const int64_t cap = W.cap;
    R r[D], rr2 = R(0);
#pragma unroll
    for (int K = 0; K < D; ++K) {
        r[K] = (R)(xj[K] - xi[K]);
        rr2 += r[K] * r[K];
    }
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) wout[cc] = R(0);
    if (rr2 == R(0)) return;
    R rr = sqrt(rr2), w, dw;
    kern_wdw<R>(rr, (R)P.inv_l, (R)P.ad, w, dw);
    R fac = -dw / rr, gt[D], rg = R(0);
#pragma unroll
    for (int K = 0; K < D; ++K) {
        R s2 = R(0);
#pragma unroll
        for (int L2 = 0; L2 < D; ++L2) s2 += (R)W.L[(int64_t)(K * D + L2) * cap + i] * fac * r[L2];
        gt[K] = s2;
        rg += r[K] * s2;
    }
    R F = rg / (rr2 * rr2), q[M];
    qvec<D, R>(r, q);
    const R V = (R)vol_of(P, c, j);
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) {
        R bq = R(0), gg = R(0);
#pragma unroll
        for (int a = 0; a < M; ++a) bq += (R)W.adj[(int64_t)(cc * S + a) * cap + i] * q[a];
#pragma unroll
        for (int K = 0; K < D; ++K) gg += gt[K] * (R)W.adj[(int64_t)(cc * S + M + K) * cap + i];
        wout[cc] = V * (F * bq + gg);
    }
}

template <int D, typename R, int NC>
__global__ void __launch_bounds__(128) k_sph2_adjm2(DevParams P, const Part c, Work W, int n,
                                                    double *phibar)
{
    int jdx = blockIdx.x * blockDim.x + threadIdx.x;
    if (jdx >= n) return;
    const int o = c.orig[jdx];
    const int tj = c.type[jdx];
    if (tj == VIRTUAL) {
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) phibar[(int64_t)cc * n + o] = 0.0;
        return;
    }
    const int64_t cap = W.cap;
    double xj[3];
    load_hat<D>(c, jdx, xj);
    Acc<R> acc[NC];
    R wv[NC];
    const int cnt = W.nbr_cnt[jdx];
    for (int k = 0; k < cnt; ++k) {
        const int i = W.nbr[(int64_t)k * cap + jdx];
        const int ti = c.type[i];
        if (ti == VIRTUAL) continue;
        double xi[3];
        load_hat<D>(c, i, xi);
        if (ti == FLUID) {   // incoming w_ij
            adj_pair_m<D, R, NC>(P, c, W, i, jdx, xi, xj, wv);
#pragma unroll
            for (int cc = 0; cc < NC; ++cc) acc[cc].add(wv[cc]);
        }
        if (tj == FLUID) {   // outgoing w_ji
            adj_pair_m<D, R, NC>(P, c, W, jdx, i, xj, xi, wv);
#pragma unroll
            for (int cc = 0; cc < NC; ++cc) acc[cc].add(-wv[cc]);
        }
    }
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) phibar[(int64_t)cc * n + o] = (double)acc[cc].val();
}

template <int D, typename R, int NC>
static void launch_sph2_adjm(const DevParams &P, Part cur, Work W, int64_t n, const double *gbar,
                             const double *d2bar, const double *lapbar, double *phibar,
                             cudaStream_t st)
{
    const unsigned g = (unsigned)((n + 127) / 128);
    k_sph2_adjm1<D, R, NC><<<g, 128, 0, st>>>(P, cur, W, (int)n, gbar, d2bar, lapbar);
    k_sph2_adjm2<D, R, NC><<<g, 128, 0, st>>>(P, cur, W, (int)n, phibar);
}

template <int D, typename R>
static void launch_sph2_adjm_nc(const DevParams &P, Part cur, Work W, int64_t n, int ncomp,
                                const double *gbar, const double *d2bar, const double *lapbar,
                                double *phibar, cudaStream_t st)
{
    if (ncomp == 1) launch_sph2_adjm<D, R, 1>(P, cur, W, n, gbar, d2bar, lapbar, phibar, st);
    else if (ncomp == 2) launch_sph2_adjm<D, R, 2>(P, cur, W, n, gbar, d2bar, lapbar, phibar, st);
    else launch_sph2_adjm<D, R, 3>(P, cur, W, n, gbar, d2bar, lapbar, phibar, st);
}

void launch_sph2_adjoint(const DevParams &P, Part cur, Work W, int64_t n, int ncomp,
                         const double *gbar, const double *d2bar, const double *lapbar,
                         double *phibar, cudaStream_t st)
{
    if (ncomp <= 3) {   // all fields in one pair of launches
        if (P.dim == 2) {
            if (P.precision == VCT_MIXED) launch_sph2_adjm_nc<2, float>(P, cur, W, n, ncomp, gbar, d2bar, lapbar, phibar, st);
            else launch_sph2_adjm_nc<2, double>(P, cur, W, n, ncomp, gbar, d2bar, lapbar, phibar, st);
        } else {
            if (P.precision == VCT_MIXED) launch_sph2_adjm_nc<3, float>(P, cur, W, n, ncomp, gbar, d2bar, lapbar, phibar, st);
            else launch_sph2_adjm_nc<3, double>(P, cur, W, n, ncomp, gbar, d2bar, lapbar, phibar, st);
        }
        return;
    }
    unsigned g = (unsigned)((n + 127) / 128);
    for (int comp = 0; comp < ncomp; ++comp) {
        if (P.dim == 2) {
            if (P.precision == VCT_MIXED) {
                k_sph2_adj1<2, float><<<g, 128, 0, st>>>(P, cur, W, (int)n, gbar, d2bar, lapbar, comp);
                k_sph2_adj2<2, float><<<g, 128, 0, st>>>(P, cur, W, (int)n, phibar, comp);
            } else {
                k_sph2_adj1<2, double><<<g, 128, 0, st>>>(P, cur, W, (int)n, gbar, d2bar, lapbar, comp);
                k_sph2_adj2<2, double><<<g, 128, 0, st>>>(P, cur, W, (int)n, phibar, comp);
            }
        } else {
            if (P.precision == VCT_MIXED) {
                k_sph2_adj1<3, float><<<g, 128, 0, st>>>(P, cur, W, (int)n, gbar, d2bar, lapbar, comp);
                k_sph2_adj2<3, float><<<g, 128, 0, st>>>(P, cur, W, (int)n, phibar, comp);
            } else {
                k_sph2_adj1<3, double><<<g, 128, 0, st>>>(P, cur, W, (int)n, gbar, d2bar, lapbar, comp);
                k_sph2_adj2<3, double><<<g, 128, 0, st>>>(P, cur, W, (int)n, phibar, comp);
            }
        }
    }
}

// Adjoint of the ISPH operator set's derivatives (Table tab:case_names, Eq. sec_0th)
// for the step's reverse: g_i = L_i sum_j V_j phi_ij grad w_ij and the 0th-order
// second derivatives D_a = sum_j V_j k_a(r_ij) phi_ij (none on an isolated
// particle), lap_i = c0 g_i,z + c~ . D_i.  Pass 1 forms per fluid particle
// bbar_a = lapbar c~_a (0 when isolated) and gbar' = gbar + c0 lapbar e_z (rows [0, m)
// and [m, m + d) of W.adj); each pair (i, j) carries w_ij = V_j [bbar_i . k(r_ij) +
// (L_i grad w_ij) . gbar'_i], gathered as for the SPH(2) operator.  FP64.
template <int D>
__global__ void __launch_bounds__(128) k_isph_adj1(DevParams P, const Part c, Work W, int n,
                                                   const double *gbar, const double *lapbar,
                                                   int comp)
{
    constexpr int M = D == 2 ? 3 : 6;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t cap = W.cap;
    if (c.type[i] != FLUID) {
        for (int a = 0; a < M + D; ++a) W.adj[(int64_t)a * cap + i] = 0.0;
        return;
    }
    const int o = c.orig[i];
    const double lb = lapbar ? lapbar[(int64_t)comp * n + o] : 0.0;
    double ct[M];
    ctilde<D>(c.c3[i], c.sx[i], c.sy[i], ct);
    const double ds = W.fs[i] == 2 ? 0.0 : 1.0;
#pragma unroll
    for (int a = 0; a < M; ++a) W.adj[(int64_t)a * cap + i] = ds * ct[a] * lb;
#pragma unroll
    for (int K = 0; K < D; ++K) {
        double gb = gbar ? gbar[((int64_t)comp * D + K) * n + o] : 0.0;
        if (K == D - 1) gb += c.c0[i] * lb;
        W.adj[(int64_t)(M + K) * cap + i] = gb;
    }
}

template <int D>
__device__ __forceinline__ double adj_pair_isph(const DevParams &P, const Part &c, const Work &W,
                                                int i, int j, const double *xi, const double *xj)
{
    constexpr int M = D == 2 ? 3 : 6;
    const int64_t cap = W.cap;
    double r[D], rr2 = 0.0;
#pragma unroll
    for (int K = 0; K < D; ++K) {
        r[K] = xj[K] - xi[K];
        rr2 += r[K] * r[K];
    }
    if (rr2 == 0.0) return 0.0;
    double rr = sqrt(rr2), w, dw;
    kern_wdw<double>(rr, P.inv_l, P.ad, w, dw);
    const double fac = -dw / rr;
    double kw[M], s = 0.0;
    er_weights<D, double>(r, rr2, fac, kw);
#pragma unroll
    for (int a = 0; a < M; ++a) s += W.adj[(int64_t)a * cap + i] * kw[a];
#pragma unroll
    for (int K = 0; K < D; ++K) {
        double gt = 0.0;
#pragma unroll
        for (int L2 = 0; L2 < D; ++L2) gt += W.L[(int64_t)(K * D + L2) * cap + i] * fac * r[L2];
        s += gt * W.adj[(int64_t)(M + K) * cap + i];
    }
    return W.vol[j] * s;
}

template <int D>
__global__ void __launch_bounds__(128) k_isph_adj2(DevParams P, const Part c, Work W, int n,
                                                   double *phibar, int comp)
{
    const int jdx = blockIdx.x * blockDim.x + threadIdx.x;
    if (jdx >= n) return;
    const int o = c.orig[jdx];
    const int tj = c.type[jdx];
    if (tj == VIRTUAL) {
        phibar[(int64_t)comp * n + o] = 0.0;
        return;
    }
    const int64_t cap = W.cap;
    double xj[3], s = 0.0;
    load_hat<D>(c, jdx, xj);
    const int cnt = W.nbr_cnt[jdx];
    for (int k = 0; k < cnt; ++k) {
        const int i = W.nbr[(int64_t)k * cap + jdx];
        const int ti = c.type[i];
        if (ti == VIRTUAL) continue;
        double xi[3];
        load_hat<D>(c, i, xi);
        if (ti == FLUID) s += adj_pair_isph<D>(P, c, W, i, jdx, xi, xj);    // incoming w_ij
        if (tj == FLUID) s -= adj_pair_isph<D>(P, c, W, jdx, i, xj, xi);    // outgoing w_ji
    }
    phibar[(int64_t)comp * n + o] = s;
}

void launch_isph_adjoint(const DevParams &P, Part cur, Work W, int64_t n, int ncomp,
                         const double *gbar, const double *lapbar, double *phibar, cudaStream_t st)
{
    const unsigned g = (unsigned)((n + 127) / 128);
    for (int comp = 0; comp < ncomp; ++comp) {
        if (P.dim == 2) {
            k_isph_adj1<2><<<g, 128, 0, st>>>(P, cur, W, (int)n, gbar, lapbar, comp);
            k_isph_adj2<2><<<g, 128, 0, st>>>(P, cur, W, (int)n, phibar, comp);
        } else {
            k_isph_adj1<3><<<g, 128, 0, st>>>(P, cur, W, (int)n, gbar, lapbar, comp);
            k_isph_adj2<3><<<g, 128, 0, st>>>(P, cur, W, (int)n, phibar, comp);
        }
    }
}

// ---------------------------------------------------------------------------
// a12 (map part): derivative of the per-particle metric with respect to the
// bathymetry parameters theta = [h0, slope_x, slope_y, cos_amp, cos_len,
// amp_g, cx_g, cy_g, width_g (g < n_gauss)].  Exact forward-mode derivatives
// with dual numbers, one parameter seeded per pass, contracted with the
// caller's adjoints of (z^, J, s_x, s_y, c0, c3) and summed over particles
// (per-block partials, then a fixed-order sum).
// ---------------------------------------------------------------------------
struct Dual {
    double v, d;
    __device__ Dual() : v(0.0), d(0.0) {}
    __device__ Dual(double a, double b = 0.0) : v(a), d(b) {}
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ __forceinline__ Dual operator/(Dual a, Dual b)
{
    return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
__device__ __forceinline__ Dual dexp(Dual a) { double e = exp(a.v); return Dual(e, e * a.d); }
__device__ __forceinline__ Dual dsin(Dual a) { return Dual(sin(a.v), cos(a.v) * a.d); }
__device__ __forceinline__ Dual dcos(Dual a) { return Dual(cos(a.v), -sin(a.v) * a.d); }

// parameter k of theta as a dual (derivative 1 if k == seed)
__device__ __forceinline__ Dual theta(const DevParams &P, int k, int seed)
{
    const int G = P.n_gauss;
    double v;
    if (k == 0) v = P.h0;
    else if (k == 1) v = P.slope_x;
    else if (k == 2) v = P.slope_y;
    else if (k == 3) v = P.cos_amp;
    else if (k == 4) v = P.cos_len;
    else {
        int q = k - 5, g = q % G, w = q / G;
        v = w == 0 ? P.gamp[g] : w == 1 ? P.gcx[g] : w == 2 ? P.gcy[g] : P.gwid[g];
    }
    return Dual(v, k == seed ? 1.0 : 0.0);
}

__device__ void bathy_dual(const DevParams &P, Dual X, Dual Y, int seed, Dual h[5])
{
    Dual sx = theta(P, 1, seed), sy = theta(P, 2, seed);
    h[0] = theta(P, 0, seed) + sx * X + sy * Y;
    h[1] = sx;
    h[2] = sy;
    h[3] = Dual(0.0);
    h[4] = Dual(0.0);
    Dual ca = theta(P, 3, seed);
    if (P.cos_amp != 0.0 || seed == 3) {
        Dual k = Dual(2.0 * 3.14159265358979323846) / theta(P, 4, seed);
        Dual kx = k * X, s = dsin(kx), c = dcos(kx);
        h[0] = h[0] + ca * c;
        h[1] = h[1] - ca * k * s;
        h[3] = h[3] - ca * k * k * c;
    }
    for (int g = 0; g < P.n_gauss; ++g) {
        Dual A = theta(P, 5 + g, seed), cx = theta(P, 5 + P.n_gauss + g, seed);
        Dual cy = theta(P, 5 + 2 * P.n_gauss + g, seed), wd = theta(P, 5 + 3 * P.n_gauss + g, seed);
        Dual dx = X - cx, dy = Y - cy, is2 = Dual(1.0) / (wd * wd);
        Dual e = A * dexp(Dual(-0.5) * (dx * dx + dy * dy) * is2);
        h[0] = h[0] + e;
        h[1] = h[1] - e * dx * is2;
        h[2] = h[2] - e * dy * is2;
        h[3] = h[3] + e * (dx * dx * is2 - Dual(1.0)) * is2;
        h[4] = h[4] + e * (dy * dy * is2 - Dual(1.0)) * is2;
    }
}

// Same metric as map_metric, in dual arithmetic: out = {z^, J, s_x, s_y, c0, c3}.
// The position (X, Y, Z) and the parameter `seed` of theta may carry derivatives.
__device__ void metric_dual(const DevParams &P, Dual X, Dual Y, Dual Z, int seed, Dual out[6])
{
    Dual a(1.0), ax, ay, axx, ayy, b, bx, by, bxx, byy;
    if (P.kind == VCT_MAP_E) {
        a = Dual(P.aspect);
    } else {
        Dual h[5];
        bathy_dual(P, X, Y, seed, h);
        b = -h[0]; bx = -h[1]; by = -h[2]; bxx = -h[3]; byy = -h[4];
        if (P.kind == VCT_MAP_BFE) {
            a = Dual(P.aspect);
        } else if (P.kind == VCT_MAP_SIGMA) {
            Dual D = Dual(P.H) - h[0];
            if (D.v <= 0.0) {
                a = Dual(P.amax);
            } else {
                double ai = P.H_hat / D.v;
                if (ai < P.amin) a = Dual(P.amin);
                else if (ai > P.amax) a = Dual(P.amax);
                else {
                    Dual Hh(P.H_hat), iD = Dual(1.0) / D;
                    a = Hh * iD;
                    ax = Hh * h[1] * iD * iD;
                    ay = Hh * h[2] * iD * iD;
                    axx = Hh * (h[3] * iD * iD + Dual(2.0) * h[1] * h[1] * iD * iD * iD);
                    ayy = Hh * (h[4] * iD * iD + Dual(2.0) * h[2] * h[2] * iD * iD * iD);
                }
            }
        }
    }
    if (P.dim == 2) {  // a 2-D section has no y direction
        ay = Dual(0.0); ayy = Dual(0.0); by = Dual(0.0); byy = Dual(0.0);
    }
    Dual zeta = Z + b;
    Dual sx = ax * zeta + a * bx, sy = ay * zeta + a * by;
    out[0] = a * zeta;
    out[1] = a;
    out[2] = sx;
    out[3] = sy;
    out[4] = (axx + ayy) * zeta + Dual(2.0) * (ax * bx + ay * by) + a * (bxx + byy);
    out[5] = a * a + sx * sx + sy * sy;
}

constexpr int MAPT = 128;

// partial[k * nblk + block] = sum over the block's particles of sum_q mbar_q dm_q/dtheta_k
__global__ void __launch_bounds__(MAPT) k_map_adjoint(DevParams P, vct_state s, int n, int nparam,
                                                      const double *const *mbar, double *partial)
{
    __shared__ double red[MAPT / 32];
    const int i = blockIdx.x * MAPT + threadIdx.x;
    double bar[6] = {0, 0, 0, 0, 0, 0};
    double x = 0, y = 0, z = 0;
    const bool act = i < n;
    if (act) {
        x = s.x[i];
        y = P.dim == 3 && s.y ? s.y[i] : 0.0;
        z = s.z[i];
        for (int q = 0; q < 6; ++q) bar[q] = mbar[q] ? mbar[q][i] : 0.0;
    }
    for (int k = 0; k < nparam; ++k) {
        double c = 0.0;
        if (act) {
            Dual out[6];
            metric_dual(P, Dual(x), Dual(y), Dual(z), k, out);
            for (int q = 0; q < 6; ++q) c += bar[q] * out[q].d;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < MAPT / 32; ++w) t += red[w];
            partial[(int64_t)k * gridDim.x + blockIdx.x] = t;
        }
        __syncthreads();
    }
}

__global__ void k_map_adjoint_sum(const double *partial, int nblk, int nparam, double *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nparam) return;
    double t = 0.0;
    for (int b = 0; b < nblk; ++b) t += partial[(int64_t)k * nblk + b];
    out[k] = t;
}

int launch_map_adjoint(const DevParams &P, vct_state s, int64_t n, const double *const *mbar_dev,
                       double *partial, int64_t partial_cap, double *out, cudaStream_t st)
{
    const int nparam = 5 + 4 * P.n_gauss;
    const int nblk = (int)((n + MAPT - 1) / MAPT);
    if ((int64_t)nblk * nparam > partial_cap) return 1;
    k_map_adjoint<<<nblk, MAPT, 0, st>>>(P, s, (int)n, nparam, mbar_dev, partial);
    k_map_adjoint_sum<<<(nparam + 127) / 128, 128, 0, st>>>(partial, nblk, nparam, out);
    return 0;
}

// Derivative of the per-particle metric with respect to the particle's own
// physical position (the map's metric under moving particles): for each
// coordinate seeded in turn, pos_bar[k * n + i] = sum_q mbar_q,i dm_q,i / dx_k
// (k over x, z in 2-D; x, y, z in 3-D).  The projected position's x^ = x and
// y^ = y parts are the identity and are not included.
__global__ void __launch_bounds__(MAPT) k_map_pos_adjoint(DevParams P, vct_state s, int n,
                                                          const double *const *mbar, double *pos_bar)
{
    const int i = blockIdx.x * MAPT + threadIdx.x;
    if (i >= n) return;
    const double x = s.x[i], y = P.dim == 3 && s.y ? s.y[i] : 0.0, z = s.z[i];
    double bar[6];
    for (int q = 0; q < 6; ++q) bar[q] = mbar[q] ? mbar[q][i] : 0.0;
    const int naxes = P.dim == 3 ? 3 : 2;
    for (int k = 0; k < naxes; ++k) {
        const int axis = P.dim == 3 ? k : (k == 0 ? 0 : 2);   // 2-D: x and z
        Dual out[6];
        metric_dual(P, Dual(x, axis == 0 ? 1.0 : 0.0), Dual(y, axis == 1 ? 1.0 : 0.0),
                    Dual(z, axis == 2 ? 1.0 : 0.0), -1, out);
        double c = 0.0;
        for (int q = 0; q < 6; ++q) c += bar[q] * out[q].d;
        pos_bar[(int64_t)k * n + i] = c;
    }
}

void launch_map_pos_adjoint(const DevParams &P, vct_state s, int64_t n, const double *const *mbar_dev,
                            double *pos_bar, cudaStream_t st)
{
    k_map_pos_adjoint<<<(unsigned)((n + MAPT - 1) / MAPT), MAPT, 0, st>>>(P, s, (int)n, mbar_dev, pos_bar);
}

// ---------------------------------------------------------------------------
// a12 (loss): water level at wave gauges (the paper's experiments record water
// levels at fixed gauges, Sec. 4.4.2).  At gauge g the free-surface fluid
// particles' heights are averaged with the weights w = spline(|r_h| / l) of
// their horizontal distance to the gauge (support 2 l); eta_g = that average
// minus the still-water level H (0 without a surface particle within 2 l), and
// the loss is sum_g eta_g^2.  Its gradient with respect to each surface
// particle's position: z_bar = sum_g 2 eta_g w / S_g, and along the horizontal
// axes 2 eta_g (z - level_g) (dw/dx) / S_g, S_g = sum w.  Caller order; the
// free-surface flags are the caller's (frozen).
// ---------------------------------------------------------------------------
constexpr int GAUGE_MAX = 16;

__device__ __forceinline__ void gauge_w(double r, double inv_l, double &w, double &dwdr)
{
    const double q = r * inv_l;
    if (q < 1.0) {
        w = 1.0 - 1.5 * q * q + 0.75 * q * q * q;
        dwdr = (-3.0 * q + 2.25 * q * q) * inv_l;
    } else if (q < 2.0) {
        const double t = 2.0 - q;
        w = 0.25 * t * t * t;
        dwdr = -0.75 * t * t * inv_l;
    } else {
        w = 0.0;
        dwdr = 0.0;
    }
}

// partial[(2 g + 0/1) * nblk + block] = the block's sum of w z / w for gauge g
__global__ void __launch_bounds__(MAPT) k_gauge_partials(DevParams P, vct_state s, int n,
                                                          const int32_t *fs, int ng,
                                                          const double *gxy, double *partial)
{
    __shared__ double red[MAPT / 32];
    const int i = blockIdx.x * MAPT + threadIdx.x;
    const bool act = i < n && fs[i] == 1 && s.type[i] == FLUID;
    const double x = act ? s.x[i] : 0.0, z = act ? s.z[i] : 0.0;
    const double y = act && P.dim == 3 ? s.y[i] : 0.0;
    for (int q = 0; q < 2 * ng; ++q) {
        const int g = q >> 1;
        double c = 0.0;
        if (act) {
            const double dx = x - gxy[2 * g], dy = P.dim == 3 ? y - gxy[2 * g + 1] : 0.0;
            double w, dwdr;
            gauge_w(sqrt(dx * dx + dy * dy), P.inv_l, w, dwdr);
            c = (q & 1) ? w : w * z;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < MAPT / 32; ++w) t += red[w];
            partial[(int64_t)q * gridDim.x + blockIdx.x] = t;
        }
        __syncthreads();
    }
}

// res[0..ng) level, res[ng..2ng) S_g, res[2ng..3ng) eta, res[3ng] the loss
__global__ void k_gauge_final(DevParams P, const double *partial, int nblk, int ng, double *res)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double loss = 0.0;
    for (int g = 0; g < ng; ++g) {
        double num = 0.0, den = 0.0;
        for (int b = 0; b < nblk; ++b) {
            num += partial[(int64_t)(2 * g) * nblk + b];
            den += partial[(int64_t)(2 * g + 1) * nblk + b];
        }
        const double level = den > 0.0 ? num / den : 0.0;
        const double eta = den > 0.0 ? level - P.H : 0.0;
        res[g] = level;
        res[ng + g] = den;
        res[2 * ng + g] = eta;
        loss += eta * eta;
    }
    res[3 * ng] = loss;
}

__global__ void __launch_bounds__(MAPT) k_gauge_grad(DevParams P, vct_state s, int n, const int32_t *fs,
                                                     int ng, const double *gxy, const double *res,
                                                     double *pos_bar)
{
    const int i = blockIdx.x * MAPT + threadIdx.x;
    if (i >= n) return;
    const int nd = P.dim == 3 ? 3 : 2;
    double bar[3] = {0.0, 0.0, 0.0};   // x, (y,) z
    if (fs[i] == 1 && s.type[i] == FLUID) {
        const double x = s.x[i], z = s.z[i], y = P.dim == 3 ? s.y[i] : 0.0;
        for (int g = 0; g < ng; ++g) {
            const double den = res[ng + g];
            if (!(den > 0.0)) continue;
            const double dx = x - gxy[2 * g], dy = P.dim == 3 ? y - gxy[2 * g + 1] : 0.0;
            const double r = sqrt(dx * dx + dy * dy);
            double w, dwdr;
            gauge_w(r, P.inv_l, w, dwdr);
            const double f = 2.0 * res[2 * ng + g] / den;
            bar[nd - 1] += f * w;
            if (r > 0.0) {
                const double h = f * (z - res[g]) * dwdr / r;
                bar[0] += h * dx;
                if (P.dim == 3) bar[1] += h * dy;
            }
        }
    }
    for (int k = 0; k < nd; ++k) pos_bar[(int64_t)k * n + i] = bar[k];
}

int launch_gauge_loss(const DevParams &P, vct_state s, int64_t n, const int32_t *fs, int ng,
                      const double *gxy, double *partial, int64_t partial_cap, double *res,
                      double *pos_bar, cudaStream_t st)
{
    if (ng < 1 || ng > GAUGE_MAX) return 1;
    const int nblk = (int)((n + MAPT - 1) / MAPT);
    if ((int64_t)nblk * 2 * ng > partial_cap) return 2;
    k_gauge_partials<<<nblk, MAPT, 0, st>>>(P, s, (int)n, fs, ng, gxy, partial);
    k_gauge_final<<<1, 32, 0, st>>>(P, partial, nblk, ng, res);
    if (pos_bar) k_gauge_grad<<<nblk, MAPT, 0, st>>>(P, s, (int)n, fs, ng, gxy, res, pos_bar);
    return 0;
}

void launch_csr_export(const DevParams &P, Part cur, Work W, int64_t n, int64_t *row_ptr,
                       int32_t *col, int64_t col_cap, cudaStream_t st)
{
    unsigned g = (unsigned)((n + 127) / 128);
    k_csr_counts<<<g, 128, 0, st>>>(cur, W, (int)n);
    exclusive_scan<int64_t>(W.scan_tmp, row_ptr, W.row_tmp, n, st);
    if (col) k_csr_fill<<<g, 128, 0, st>>>(cur, W, (int)n, row_ptr, col, col_cap);
}

// ---------------------------------------------------------------------------
// Probe outputs (caller order)
// ---------------------------------------------------------------------------
__global__ void k_probe_out(DevParams P, const Part c, Work W, int n, vct_probe pr)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int o = c.orig[i];
    bool fl = c.type[i] == FLUID;
    if (pr.fs) pr.fs[o] = fl ? W.fs[i] : 0;
    if (pr.rho_hat) pr.rho_hat[o] = fl ? W.rho_hat[i] : 0.0;
    if (pr.nu) pr.nu[o] = fl ? W.nu[i] : 0.0;
    if (pr.lam_min) pr.lam_min[o] = fl ? W.lam[i] : 0.0;
    if (pr.vstar)
        for (int cc = 0; cc < P.dim; ++cc)
            pr.vstar[(int64_t)cc * n + o] = fl ? W.vstar[(int64_t)cc * W.cap + i] : 0.0;
    if (pr.ppe_b) pr.ppe_b[o] = W.bvec[i];
    if (pr.jbar_used) pr.jbar_used[o] = c.jbar[i];
    if (pr.vwall) {
        const bool wl = c.type[i] == WALL && P.slip;
        const double vv[3] = {c.u[i], P.dim == 3 ? c.v[i] : 0.0, c.w[i]};
        for (int cc = 0; cc < P.dim; ++cc)
            pr.vwall[(int64_t)cc * n + o] = wl ? vv[cc == P.dim - 1 ? 2 : cc] : 0.0;
    }
}

// Free-slip walls (Sec. 3.5): wall particle j carries v_j = (I - 2 n n) v_wall,j,
// v_wall,j = sum_k V_k v_k w_jk / sum_k V_k w_jk over its fluid neighbours (SPH
// interpolation; 0 without any), n the outer unit normal in physical space: the
// projected normal n^ ~ sum_{k virtual} V0 grad w_jk (towards the virtual
// particles outside the wall) transformed as a gradient, n ~ J^T n^ (on the
// bottom: the surface normal the paper builds from rotations by arctan h_x,
// arctan h_y).  Written into the sorted state (FP64 and the hi/lo FP32 copy) of
// wall particles, where pass 1, pass 2 and the right side read it.
template <int D>
__device__ __forceinline__ void wall_velocity_body(const DevParams &P, const Part &c, const Work &W, int n, int bid_)
{
    if (step_failed(W.status)) return;
    const int j = bid_ * blockDim.x + threadIdx.x;
    if (j >= n || c.type[j] != WALL) return;
    const int64_t cap = W.cap;
    double xj[3];
    load_hat<D>(c, j, xj);
    double num[3] = {0.0, 0.0, 0.0}, den = 0.0, nh[3] = {0.0, 0.0, 0.0};
    const int cnt = W.nbr_cnt[j];
    for (int q = 0; q < cnt; ++q) {
        const int k = W.nbr[(int64_t)q * cap + j];
        const int tk = c.type[k];
        if (tk == WALL) continue;
        double xk[3], r[3], rr2 = 0.0;
        load_hat<D>(c, k, xk);
#pragma unroll
        for (int K = 0; K < D; ++K) {
            r[K] = xk[K] - xj[K];
            rr2 += r[K] * r[K];
        }
        const double rr = sqrt(rr2);
        double w, dw;
        kern_wdw<double>(rr, P.inv_l, P.ad, w, dw);
        if (tk == FLUID) {
            double vk[3];
            load_vel<D>(c, k, vk);
            const double wv = vol_of(P, c, k) * w;
#pragma unroll
            for (int cc = 0; cc < D; ++cc) num[cc] += wv * vk[cc];
            den += wv;
        } else if (rr > 0.0) {
#pragma unroll
            for (int K = 0; K < D; ++K) nh[K] += P.V0 * (-dw / rr) * r[K];
        }
    }
    double v[3] = {0.0, 0.0, 0.0};
    if (den > 0.0) {
        double nn[D], nl = 0.0, vn = 0.0;
#pragma unroll
        for (int cc = 0; cc < D; ++cc) v[cc] = num[cc] / den;
        jac_apply<D>(c.J[j], c.sx[j], c.sy[j], nh, nn);
#pragma unroll
        for (int I = 0; I < D; ++I) nl += nn[I] * nn[I];
        nl = sqrt(nl);
        if (nl > 0.0) {
#pragma unroll
            for (int I = 0; I < D; ++I) {
                nn[I] /= nl;
                vn += nn[I] * v[I];
            }
#pragma unroll
            for (int cc = 0; cc < D; ++cc) v[cc] -= 2.0 * vn * nn[cc];
        }
    }
    c.u[j] = v[0];
    if (D == 3) c.v[j] = v[1];
    c.w[j] = v[D - 1];
    float4 lo;
    W.velhi[j] = f4_hilo_split(v[0], D == 3 ? v[1] : 0.0, v[D - 1], lo);
    W.vello[j] = lo;
}

template <int D>
__global__ void __launch_bounds__(128) k_wall_velocity(DevParams P, Part c, Work W, int n)
{
    wall_velocity_body<D>(P, c, W, n, blockIdx.x);
}

void launch_wall_velocity(const DevParams &P, Part cur, Work W, int64_t n, cudaStream_t st)
{
    const unsigned g = (unsigned)((n + 127) / 128);
    if (P.dim == 2) k_wall_velocity<2><<<g, 128, 0, st>>>(P, cur, W, (int)n);
    else k_wall_velocity<3><<<g, 128, 0, st>>>(P, cur, W, (int)n);
}

// Parity probes only: replace the free-surface flags pass 1 decided by the
// caller's (caller order), for fluid particles, before anything reads them.
__global__ void k_force_fs(const Part c, Work W, int n, const int32_t *fs_in)
{
    if (step_failed(W.status)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || c.type[i] != FLUID) return;
    const int32_t v = fs_in[c.orig[i]];
    W.fs[i] = v == 2 ? 2 : (v ? 1 : 0);
}

void launch_force_fs(Part cur, Work W, int64_t n, const int32_t *fs_in, cudaStream_t st)
{
    k_force_fs<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(cur, W, (int)n, fs_in);
}

void launch_probe_out(const DevParams &P, Part cur, Work W, int64_t n, const vct_probe &pr,
                      cudaStream_t st)
{
    k_probe_out<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(P, cur, W, (int)n, pr);
}

// (After a failed step the pressure rows may never have been written: the
// probe's A x then reads nothing from them and writes zeros.)
__global__ void k_gather_masked(const Part c, Work W, int n, const double *xin, double *xs)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    xs[i] = !step_failed(W.status) && W.pcnt[i] >= 0 ? xin[c.orig[i]] : 0.0;
}

__global__ void k_spmv_out(const Part c, Work W, int n, const double *xs, double *out,
                           int mixed, int dim)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int pc = step_failed(W.status) ? -1 : W.pcnt[i];
    double y = 0.0;
    if (pc >= 0) {
        y = W.diag[i] * xs[i];
        for (int k = 0; k < pc; ++k) {
            int64_t q = ell_at_dim(dim, k, i, W.cap);
            double a = mixed ? (double)W.pvalf[q] : W.pval[q];
            y += a * xs[W.pcol[q]];
        }
    }
    out[c.orig[i]] = y;
}

void launch_probe_ax(const DevParams &P, Part cur, Work W, int64_t n, const double *x_test,
                     double *out, cudaStream_t st)
{
    unsigned g = (unsigned)((n + 255) / 256);
    k_gather_masked<<<g, 256, 0, st>>>(cur, W, (int)n, x_test, W.kt);
    k_spmv_out<<<g, 256, 0, st>>>(cur, W, (int)n, W.kt, out, P.precision == VCT_MIXED, P.dim);
}

void launch_store(const DevParams &P, Part cur, vct_state s, int64_t n, const int32_t *status,
                  cudaStream_t st)
{
    k_store_w<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(P, cur, s, (int)n, status);
}


// ---------------------------------------------------------------------------
// a12 (part): adjoint of the pressure solve.  The step solves A p = b on the
// unknown rows (fluid particles off the free surface; Eqs. VCT_ppe, PNC).  For
// p = A^-1 b, a loss gradient p_bar gives b_bar = A^-T p_bar, and the
// coefficients' adjoint is A_bar = -b_bar p^T on A's pattern.
//
// A's pattern is symmetric: row i holds the unknown neighbours of i, and the
// neighbour relation is symmetric in projected space.  So row j of A^T has the
// columns of row j of A, and its coefficient in column i is row i's
// coefficient in column j; k_adj_tslot finds that slot of row i once per call
// (in the neighbour-list scratch, which the next step rebuilds).  The solve is
// BiCGSTAB (van der Vorst 1992) in FP64 with a Jacobi (diagonal) right
// preconditioner, one thread per row, in one cooperative launch; the operator
// is the one the forward solve used (FP32 coefficients in the mixed form).
// ---------------------------------------------------------------------------
__global__ void k_adj_gather(const Part c, Work W, int n, const double *p_bar)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    W.bvec[i] = W.pcnt[i] >= 0 ? p_bar[c.orig[i]] : 0.0;
    W.kx[i] = 0.0;
}

template <int D>
__global__ void k_adj_tslot(Work W, int n)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int pc = W.pcnt[j];
    const int64_t cap = W.cap;
    for (int k = 0; k < pc; ++k) {
        const int i = W.pcol[ell_at<ell_group<D>()>(k, j, cap)];
        const int pi = W.pcnt[i];
        int t = -1;
        for (int q = 0; q < pi && t < 0; ++q)
            if (W.pcol[ell_at<ell_group<D>()>(q, i, cap)] == j) t = q;
        // only a truncated neighbour list (capacity error) breaks the symmetry
        if (t < 0) set_error(W.status, VCT_ERR_CAPACITY, j);
        W.nbr[(int64_t)k * cap + j] = t;
    }
}

// (A^T x)_j for an unknown row j
template <int D, typename CT>
__device__ __forceinline__ double adj_row(const Work &W, int j, const double *x)
{
    const int64_t cap = W.cap;
    const int pc = W.pcnt[j];
    double s = W.diag[j] * __ldcg(x + j);
    for (int k = 0; k < pc; ++k) {
        const int i = W.pcol[ell_at<ell_group<D>()>(k, j, cap)];
        const int t = W.nbr[(int64_t)k * cap + j];
        if (t >= 0) s += (double)coef<CT>(W, ell_at<ell_group<D>()>(t, i, cap)) * __ldcg(x + i);
    }
    return s;
}

// Jacobi preconditioner: 1 / diag (1 where a row has no coupling at all)
__device__ __forceinline__ double adj_dinv(const Work &W, int i)
{
    const double d = W.diag[i];
    return d != 0.0 ? 1.0 / d : 1.0;
}

template <int D, typename CT>
__global__ void __launch_bounds__(KT) k_adj_bicgstab(Work W, int n, int maxit, double rtol,
                                                      int32_t *iters_out, double *resid_out)
{
    if (step_failed(W.status)) return;
    const unsigned nb = gridDim.x;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gth = gridDim.x * blockDim.x;
    const double *g = W.bvec;
    double *x = W.kx, *r = W.kf, *rh = (double *)W.kr, *p = (double *)W.kp0, *ph = (double *)W.kp1;
    double *v = (double *)W.kv0, *s = (double *)W.ks, *sh = (double *)W.kv1, *t = (double *)W.kt;
    // r = g (x = 0), rh = r, p = r, ph = D^-1 p; |g|^2
    double part[1] = {0.0};
    for (int i = gtid; i < n; i += gth) {
        if (W.pcnt[i] < 0) continue;
        const double gi = g[i];
        r[i] = gi;
        rh[i] = gi;
        p[i] = gi;
        ph[i] = gi * adj_dinv(W, i);
        part[0] += gi * gi;
    }
    block_partials<1>(part, W.partial);
    if (!grid_barrier(W.bar, nb, W.status, blockIdx.x, W.spin_limit)) return;
    double tot[1];
    grid_totals<1>(W.partial, nb, tot);
    const double bn = sqrt(tot[0]);
    double rho = tot[0], rn = bn;
    int it = 0;
    bool fail = false;
    while (bn > 0.0 && rn > rtol * bn) {
        if (it >= maxit) {
            fail = true;
            break;
        }
        ++it;
        // v = A^T ph; (rh, v)
        double pv[1] = {0.0};
        for (int i = gtid; i < n; i += gth) {
            if (W.pcnt[i] < 0) continue;
            const double vi = adj_row<D, CT>(W, i, ph);
            v[i] = vi;
            pv[0] += rh[i] * vi;
        }
        block_partials<1>(pv, W.partial);
        if (!grid_barrier(W.bar, nb, W.status, blockIdx.x, W.spin_limit)) return;
        grid_totals<1>(W.partial, nb, tot);
        if (tot[0] == 0.0) {
            fail = true;
            break;
        }
        const double alpha = rho / tot[0];
        // s = r - alpha v, sh = D^-1 s
        for (int i = gtid; i < n; i += gth) {
            if (W.pcnt[i] < 0) continue;
            const double si = r[i] - alpha * v[i];
            s[i] = si;
            sh[i] = si * adj_dinv(W, i);
        }
        if (!grid_barrier(W.bar, nb, W.status, blockIdx.x, W.spin_limit)) return;
        // t = A^T sh; (t, s), (t, t), (s, s), (rh, s), (rh, t)
        double q[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (int i = gtid; i < n; i += gth) {
            if (W.pcnt[i] < 0) continue;
            const double ti = adj_row<D, CT>(W, i, sh), si = s[i], hi = rh[i];
            t[i] = ti;
            q[0] += ti * si;
            q[1] += ti * ti;
            q[2] += si * si;
            q[3] += hi * si;
            q[4] += hi * ti;
        }
        block_partials<5>(q, W.partial);
        if (!grid_barrier(W.bar, nb, W.status, blockIdx.x, W.spin_limit)) return;
        double tq[5];
        grid_totals<5>(W.partial, nb, tq);
        const double omega = tq[1] > 0.0 ? tq[0] / tq[1] : 0.0;
        const double rho_new = tq[3] - omega * tq[4];
        rn = sqrt(fmax(tq[2] - 2.0 * omega * tq[0] + omega * omega * tq[1], 0.0));
        if (omega == 0.0 || rho_new == 0.0) {   // the update below still applies alpha
            fail = rn > rtol * bn;
        }
        const double beta = (rho_new / rho) * (alpha / (omega != 0.0 ? omega : 1.0));
        // x += alpha ph + omega sh; r = s - omega t; p = r + beta (p - omega v); ph = D^-1 p
        for (int i = gtid; i < n; i += gth) {
            if (W.pcnt[i] < 0) continue;
            x[i] += alpha * ph[i] + omega * sh[i];
            const double ri = s[i] - omega * t[i];
            r[i] = ri;
            const double pi = ri + beta * (p[i] - omega * v[i]);
            p[i] = pi;
            ph[i] = pi * adj_dinv(W, i);
        }
        rho = rho_new;
        if (!grid_barrier(W.bar, nb, W.status, blockIdx.x, W.spin_limit)) return;
        if (omega == 0.0 || rho_new == 0.0) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (fail) set_error(W.status, VCT_ERR_NOCONV, -1);
        iters_out[0] += it;
        if (it > iters_out[1]) iters_out[1] = it;
        iters_out[2] = it;
        *resid_out = bn > 0.0 ? rn / bn : 0.0;
    }
}

__global__ void k_adj_scatter(const Part c, Work W, int n, double *b_bar)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    b_bar[c.orig[i]] = W.pcnt[i] >= 0 ? W.kx[i] : 0.0;
}

static const void *adj_fn(int precision, int dim)
{
    if (precision == VCT_MIXED)
        return dim == 2 ? (const void *)k_adj_bicgstab<2, float> : (const void *)k_adj_bicgstab<3, float>;
    return dim == 2 ? (const void *)k_adj_bicgstab<2, double> : (const void *)k_adj_bicgstab<3, double>;
}

// A^T in place of A.  The pattern is symmetric (row i holds the unknown
// neighbours of i, the neighbour relation is symmetric), so A^T has A's pattern,
// and its coefficient in row j, column i is A's in row i, column j: with the
// transposed-slot table of k_adj_tslot (in the neighbour-list scratch) each pair
// of coefficients is swapped once, by the row with the smaller index.  A second
// pass restores A.
template <int D, typename T>
__global__ void k_ell_transpose(Work W, int n, T *vals)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int pc = W.pcnt[j];
    const int64_t cap = W.cap;
    for (int k = 0; k < pc; ++k) {
        const int64_t q = ell_at<ell_group<D>()>(k, j, cap);
        const int i = W.pcol[q];
        if (i <= j) continue;
        const int t = W.nbr[(int64_t)k * cap + j];
        if (t < 0) continue;
        const int64_t qt = ell_at<ell_group<D>()>(t, i, cap);
        const T a = vals[q];
        vals[q] = vals[qt];
        vals[qt] = a;
    }
}

void launch_ppe_transpose(const DevParams &P, Work W, int64_t n, bool build_slots, cudaStream_t st)
{
    const unsigned g = (unsigned)((n + 255) / 256);
    if (build_slots) {
        if (P.dim == 2) k_adj_tslot<2><<<g, 256, 0, st>>>(W, (int)n);
        else k_adj_tslot<3><<<g, 256, 0, st>>>(W, (int)n);
    }
    if (P.precision == VCT_MIXED) {
        if (P.dim == 2) k_ell_transpose<2, float><<<g, 256, 0, st>>>(W, (int)n, W.pvalf);
        else k_ell_transpose<3, float><<<g, 256, 0, st>>>(W, (int)n, W.pvalf);
    } else {
        if (P.dim == 2) k_ell_transpose<2, double><<<g, 256, 0, st>>>(W, (int)n, W.pval);
        else k_ell_transpose<3, double><<<g, 256, 0, st>>>(W, (int)n, W.pval);
    }
}

void launch_adj_gather(Part cur, Work W, int64_t n, const double *p_bar, cudaStream_t st)
{
    k_adj_gather<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(cur, W, (int)n, p_bar);
}

void launch_adj_scatter(Part cur, Work W, int64_t n, double *b_bar, cudaStream_t st)
{
    k_adj_scatter<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(cur, W, (int)n, b_bar);
}

int launch_ppe_adjoint(const DevParams &P, Part cur, Work W, int64_t n, const double *p_bar,
                       double *b_bar, cudaStream_t st)
{
    const unsigned g = (unsigned)((n + 255) / 256);
    k_adj_gather<<<g, 256, 0, st>>>(cur, W, (int)n, p_bar);
    if (P.dim == 2) k_adj_tslot<2><<<g, 256, 0, st>>>(W, (int)n);
    else k_adj_tslot<3><<<g, 256, 0, st>>>(W, (int)n);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void *fn = adj_fn(P.precision, P.dim);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, KT, 0);
    if (per > 2) per = 2;
    int64_t want = (n + KT - 1) / KT;
    int nblk = sms * per;
    if (nblk > PSTRIDE) nblk = PSTRIDE;
    if (want < nblk) nblk = (int)want;
    if (nblk < 1) nblk = 1;
    int nn = (int)n, maxit = P.max_iter;
    double rtol = P.rtol;
    int32_t *it_out = W.kiters;
    double *res_out = W.kresid;
    void *args[] = {(void *)&W, (void *)&nn, (void *)&maxit, (void *)&rtol, (void *)&it_out,
                    (void *)&res_out};
    cudaMemsetAsync(W.bar, 0, 2 * sizeof(unsigned int), st);
    cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(nblk), dim3(KT), args, 0, st);
    if (e != cudaSuccess) return (int)e;
    k_adj_scatter<<<g, 256, 0, st>>>(cur, W, (int)n, b_bar);
    return 0;
}

// ---------------------------------------------------------------------------
// a12 (part): reverse of one time step with respect to the fluid velocities
// (Eqs. VCT_predictor, VCT_ppe, PNC, VCT_update), positions held at the start
// of the step.  With the positions fixed the step is affine in v^N:
//   f_i   = nu lap(v)_i + g                        (predictor, Eq. lap_VCT)
//   v*_i  = v_i + dt f_i
//   b_i   = rho/dt tr(J L_i X_i) - w_i . f_i + c   (X_i[c][K] = sum_j V_j (v_j - v*_i)_c fac r_K,
//                                                   a wall j carrying v_wall + dt f_i; w_i: the
//                                                   wall coefficients of Eq. PNC, W.pwall)
//   p     = A^-1 b                                 (unknown rows: fluid off the free surface)
//   v'_i  = v*_i - dt/rho J L_i sum_j V_j fac r p_ij,  p_ij = p_j - p_i or rho (r_j - r_i)_phys . f_i
//   x'_i  = x_i + dt v'_i
// so its adjoint is the transposed chain, run backwards: u = v'_bar + dt x'_bar,
// a_i = L_i^T J^T (-dt/rho u_i), then p_bar (gathers over the symmetric neighbour
// relation), b_bar = A^-T p_bar, the right side's adjoint (Y_i = rho/dt b_bar_i J L_i
// per unknown row), f_bar, and the viscous term's adjoint (the SPH(2) derivative
// operator's, with lap_bar = nu f_bar).  W.sadj rows: a [0, d), v*_bar [d, 2d),
// f_bar [2d, 3d), Y [3d, 3d + d^2); W.sadj_co: p_bar, b_bar, lap_bar (d rows), all
// caller order with stride n.
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void jac_apply_t(double J, double sx, double sy, const double *g,
                                            double *gh)
{
    // gh = J_m^T g for the Jacobian applied by jac_apply
    if (D == 2) {
        gh[0] = g[0];
        gh[1] = sx * g[0] + J * g[1];
    } else {
        gh[0] = g[0];
        gh[1] = g[1];
        gh[2] = sx * g[0] + sy * g[1] + J * g[2];
    }
}

__device__ __forceinline__ bool pp_unknown(const Part &c, const Work &W, int i)
{
    return c.type[i] == FLUID && !W.fs[i];
}

// -dw/r of the pair at separation r (projected), or 0 for coincident particles;
// in the mixed form's arithmetic (FP32 there, the separation formed in FP64 first)
template <int D>
__device__ __forceinline__ double pair_fac(const DevParams &P, const double *r)
{
    double rr2 = 0.0;
#pragma unroll
    for (int K = 0; K < D; ++K) rr2 += r[K] * r[K];
    if (rr2 == 0.0) return 0.0;
    if (P.precision == VCT_MIXED) {
        const float rr = sqrtf((float)rr2);
        float w, dw;
        kern_wdw<float>(rr, (float)P.inv_l, (float)P.ad, w, dw);
        return (double)(-dw / rr);
    }
    double rr = sqrt(rr2), w, dw;
    kern_wdw<double>(rr, P.inv_l, P.ad, w, dw);
    return -dw / rr;
}

// Corrector: u, a_i = L_i^T J^T (-dt/rho u_i) (SUM, the ISPH summation gradient
// sum_j V_j (p_ij + 2 p_i) grad w_ij: J^T (-dt/rho u_i), no L), v*_bar = u, f_bar from
// the wall pairs p_ij = rho (r_j - r_i)_phys . f_i.
template <int D, bool SUM>
__global__ void __launch_bounds__(128) k_stepadj_corr(DevParams P, const Part c, Work W, int n,
                                                      const double *v_bar, const double *x_bar)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t cap = W.cap;
    double *S = W.sadj;
    if (c.type[i] != FLUID) {
#pragma unroll
        for (int k = 0; k < 3 * D; ++k) S[(int64_t)k * cap + i] = 0.0;
        return;
    }
    const int o = c.orig[i];
    double u[D], g[D], gh[D], a[D];
#pragma unroll
    for (int cc = 0; cc < D; ++cc) {
        u[cc] = (v_bar ? v_bar[(int64_t)cc * n + o] : 0.0) +
                (x_bar ? P.dt * x_bar[(int64_t)cc * n + o] : 0.0);
        g[cc] = -P.dt / P.rho * u[cc];
    }
    jac_apply_t<D>(c.J[i], c.sx[i], c.sy[i], g, gh);
#pragma unroll
    for (int K = 0; K < D; ++K) {
        double s = 0.0;
#pragma unroll
        for (int L2 = 0; L2 < D; ++L2) s += W.L[(int64_t)(L2 * D + K) * cap + i] * gh[L2];
        a[K] = SUM ? gh[K] : s;
    }
    double xi[3], pi_[3], fb[D];
    load_hat<D>(c, i, xi);
    load_phys<D>(c, i, pi_);
#pragma unroll
    for (int K = 0; K < D; ++K) fb[K] = 0.0;
    const int cnt = W.nbr_cnt[i];
    for (int k = 0; k < cnt; ++k) {
        const int j = W.nbr[(int64_t)k * cap + i];
        const int tj = c.type[j];
        if (tj == VIRTUAL || tj == FLUID) continue;
        double xj[3], pj[3], r[D], ra = 0.0;
        load_hat<D>(c, j, xj);
        load_phys<D>(c, j, pj);
#pragma unroll
        for (int K = 0; K < D; ++K) {
            r[K] = xj[K] - xi[K];
            ra += r[K] * a[K];
        }
        const double e = P.rho * W.vol[j] * pair_fac<D>(P, r) * ra;
#pragma unroll
        for (int K = 0; K < D; ++K) fb[K] += e * (pj[K] - pi_[K]);
    }
#pragma unroll
    for (int K = 0; K < D; ++K) {
        S[(int64_t)K * cap + i] = a[K];
        S[(int64_t)(D + K) * cap + i] = u[K];
        S[(int64_t)(2 * D + K) * cap + i] = fb[K];
    }
}

// p_bar_k = p_bar_in + sum_{i fluid in S_k} [V_k fac (r_ik . a_i) + V_i fac (r_ik . a_k)]
// on unknown rows (r_ik = x^_k - x^_i), 0 elsewhere; caller order.  SUM: the summation
// gradient's 2 p_k sum_j V_j grad w_kj adds -2 V_j fac (r_jk . a_k) over every fluid and
// wall neighbour j.
template <int D, bool SUM>
__global__ void __launch_bounds__(128) k_stepadj_pbar(DevParams P, const Part c, Work W, int n,
                                                      const double *p_bar)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t cap = W.cap;
    const int o = c.orig[k];
    double *pb = W.sadj_co;
    if (!pp_unknown(c, W, k)) {
        pb[o] = 0.0;
        return;
    }
    double xk[3], ak[D];
    load_hat<D>(c, k, xk);
#pragma unroll
    for (int K = 0; K < D; ++K) ak[K] = W.sadj[(int64_t)K * cap + k];
    const double Vk = W.vol[k];
    double s = p_bar ? p_bar[o] : 0.0;
    const int cnt = W.nbr_cnt[k];
    for (int q = 0; q < cnt; ++q) {
        const int i = W.nbr[(int64_t)q * cap + k];
        const int ti = c.type[i];
        if (ti == VIRTUAL || (!SUM && ti != FLUID)) continue;
        double xi[3], r[D], rai = 0.0, rak = 0.0;
        load_hat<D>(c, i, xi);
#pragma unroll
        for (int K = 0; K < D; ++K) {
            r[K] = xk[K] - xi[K];
            rai += r[K] * W.sadj[(int64_t)K * cap + i];
            rak += r[K] * ak[K];
        }
        const double fac = pair_fac<D>(P, r), Vi = W.vol[i];
        if (ti == FLUID) s += fac * (Vk * rai + Vi * rak);
        if (SUM) s -= 2.0 * fac * Vi * rak;
    }
    pb[o] = s;
}

// Right side, own terms of each unknown row i (b_bar_i from the transposed solve):
// Y = rho/dt b_bar J L_i; v*_bar_i -= sum_j V_j fac (Y r); f_bar_i += dt sum_walls
// V_j fac (Y r) - b_bar w_i.
template <int D>
__global__ void __launch_bounds__(128) k_stepadj_rhs(DevParams P, const Part c, Work W, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t cap = W.cap;
    double *S = W.sadj;
    if (!pp_unknown(c, W, i)) {
#pragma unroll
        for (int k = 0; k < D * D; ++k) S[(int64_t)(3 * D + k) * cap + i] = 0.0;
        return;
    }
    const double bb = W.sadj_co[(int64_t)n + c.orig[i]];
    double Y[D * D];
#pragma unroll
    for (int Lc = 0; Lc < D; ++Lc) {   // column Lc of J L_i
        double col[D], jc[D];
#pragma unroll
        for (int K = 0; K < D; ++K) col[K] = W.L[(int64_t)(K * D + Lc) * cap + i];
        jac_apply<D>(c.J[i], c.sx[i], c.sy[i], col, jc);
#pragma unroll
        for (int cc = 0; cc < D; ++cc) Y[cc * D + Lc] = P.rho / P.dt * bb * jc[cc];
    }
    double xi[3], vb[D], fb[D];
    load_hat<D>(c, i, xi);
#pragma unroll
    for (int cc = 0; cc < D; ++cc) {
        vb[cc] = S[(int64_t)(D + cc) * cap + i];
        fb[cc] = S[(int64_t)(2 * D + cc) * cap + i] - bb * W.pwall[(int64_t)cc * cap + i];
    }
    const int cnt = W.nbr_cnt[i];
    for (int k = 0; k < cnt; ++k) {
        const int j = W.nbr[(int64_t)k * cap + i];
        const int tj = c.type[j];
        if (tj == VIRTUAL) continue;
        double xj[3], r[D];
        load_hat<D>(c, j, xj);
#pragma unroll
        for (int K = 0; K < D; ++K) r[K] = xj[K] - xi[K];
        const double w = W.vol[j] * pair_fac<D>(P, r);
#pragma unroll
        for (int cc = 0; cc < D; ++cc) {
            double t = 0.0;
#pragma unroll
            for (int K = 0; K < D; ++K) t += Y[cc * D + K] * r[K];
            vb[cc] -= w * t;
            if (tj != FLUID) fb[cc] += P.dt * w * t;
        }
    }
#pragma unroll
    for (int k = 0; k < D * D; ++k) S[(int64_t)(3 * D + k) * cap + i] = Y[k];
#pragma unroll
    for (int cc = 0; cc < D; ++cc) {
        S[(int64_t)(D + cc) * cap + i] = vb[cc];
        S[(int64_t)(2 * D + cc) * cap + i] = fb[cc];
    }
}

// Right side, neighbour terms (the transpose as a gather): v*_bar_j += sum over
// unknown k in S_j of V_j fac (Y_k r_kj); then f_bar_j += dt v*_bar_j and
// lap_bar_j = nu_j f_bar_j (caller order) for the viscous term's adjoint.
template <int D>
__global__ void __launch_bounds__(128) k_stepadj_gather(DevParams P, const Part c, Work W, int n)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int64_t cap = W.cap;
    double *S = W.sadj;
    const int o = c.orig[j];
    double *lb = W.sadj_co + 2 * (int64_t)n;
    const int tj = c.type[j];
#pragma unroll
    for (int cc = 0; cc < D; ++cc) lb[(int64_t)cc * n + o] = 0.0;
    // a free-slip wall particle's velocity enters the right side like a fluid
    // particle's (its v_j - v*_i); it gathers the same terms
    if (tj == VIRTUAL || (tj == WALL && !P.slip)) return;
    double xj[3], vb[D];
    load_hat<D>(c, j, xj);
#pragma unroll
    for (int cc = 0; cc < D; ++cc) vb[cc] = S[(int64_t)(D + cc) * cap + j];
    const double Vj = W.vol[j];
    const int cnt = W.nbr_cnt[j];
    for (int q = 0; q < cnt; ++q) {
        const int k = W.nbr[(int64_t)q * cap + j];
        if (!pp_unknown(c, W, k)) continue;
        double xk[3], r[D];
        load_hat<D>(c, k, xk);
#pragma unroll
        for (int K = 0; K < D; ++K) r[K] = xj[K] - xk[K];
        const double w = Vj * pair_fac<D>(P, r);
#pragma unroll
        for (int cc = 0; cc < D; ++cc) {
            double t = 0.0;
#pragma unroll
            for (int K = 0; K < D; ++K) t += S[(int64_t)(3 * D + cc * D + K) * cap + k] * r[K];
            vb[cc] += w * t;
        }
    }
#pragma unroll
    for (int cc = 0; cc < D; ++cc) S[(int64_t)(D + cc) * cap + j] = vb[cc];
    if (tj != FLUID) return;
    const double nu = W.nu[j];
#pragma unroll
    for (int cc = 0; cc < D; ++cc) {
        const double fb = S[(int64_t)(2 * D + cc) * cap + j] + P.dt * vb[cc];   // f_bar, final
        S[(int64_t)(2 * D + cc) * cap + j] = fb;
        lb[(int64_t)cc * n + o] = nu * fb;
    }
}

// The velocity field the step's viscous term differentiates (fluid velocities,
// and the free-slip wall velocities where on), in caller order for the SPH(2)
// operator: phi_co[c n + orig].
template <int D>
__global__ void k_stepadj_vcopy(const Part c, Work W, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v[3];
    load_vel<D>(c, i, v);
    double *phi = W.sadj_co + (2 + D) * (int64_t)n;
    const int o = c.orig[i];
#pragma unroll
    for (int cc = 0; cc < D; ++cc) phi[(int64_t)cc * n + o] = c.type[i] == VIRTUAL ? 0.0 : v[cc];
}

// Eddy viscosity (Sec. 3.4), first part, per fluid particle j with its final
// f_bar: the step has f = nu lap + T + g, T_c = sum_J (G_cJ + G_Jc) gn_J with
// G_IJ = dv_J/dx_I, gn = J L sum_k V_k (nu_k - nu_j) grad w_jk, nu = nu_K + nu_E.
// Writes nu_bar_j = f_bar . lap - (its own share of gn's sum), G_bar from T, and
// b_j = L^T J^T gn_bar for the neighbours' share (k_stepadj_smag2).
// W.sadj rows: b [3d + d^2, 4d + d^2), nu_bar 4d + d^2, G_bar [4d + d^2 + 1, 4d + 2 d^2 + 1).
template <int D>
__global__ void __launch_bounds__(128) k_stepadj_smag1(DevParams P, const Part c, Work W, int n)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n || c.type[j] != FLUID) return;
    const int64_t cap = W.cap;
    double *S = W.sadj;
    const int RB = 3 * D + D * D, RN = RB + D, RG = RN + 1;
    const int o = c.orig[j];
    const double *lap = W.sadj_co + (2 + 2 * D) * (int64_t)n;
    double G[D * D], fb[D];
#pragma unroll
    for (int cc = 0; cc < D; ++cc) {
        double gh[D], g[D];
#pragma unroll
        for (int K = 0; K < D; ++K) gh[K] = W.gv[(int64_t)(cc * D + K) * cap + j];
        jac_apply<D>(c.J[j], c.sx[j], c.sy[j], gh, g);
#pragma unroll
        for (int I = 0; I < D; ++I) G[I * D + cc] = g[I];
        fb[cc] = S[(int64_t)(2 * D + cc) * cap + j];
    }
    // gn (forward) from the neighbours' viscosities
    double xj[3], gs[D];
    load_hat<D>(c, j, xj);
#pragma unroll
    for (int K = 0; K < D; ++K) gs[K] = 0.0;
    const double nuj = W.nu[j];
    const int cnt = W.nbr_cnt[j];
    for (int q = 0; q < cnt; ++q) {
        const int k = W.nbr[(int64_t)q * cap + j];
        const int tk = c.type[k];
        if (tk == VIRTUAL) continue;
        double xk[3], r[D];
        load_hat<D>(c, k, xk);
#pragma unroll
        for (int K = 0; K < D; ++K) r[K] = xk[K] - xj[K];
        const double e = W.vol[k] * ((tk == FLUID ? W.nu[k] : P.nu_k) - nuj) * pair_fac<D>(P, r);
#pragma unroll
        for (int K = 0; K < D; ++K) gs[K] += e * r[K];
    }
    double gnh[D], gn[D];
#pragma unroll
    for (int K = 0; K < D; ++K) {
        double s = 0.0;
#pragma unroll
        for (int L2 = 0; L2 < D; ++L2) s += W.L[(int64_t)(K * D + L2) * cap + j] * gs[L2];
        gnh[K] = s;
    }
    jac_apply<D>(c.J[j], c.sx[j], c.sy[j], gnh, gn);
    // T's adjoint
    double Gb[D * D], gnb[D], nub = 0.0;
#pragma unroll
    for (int k = 0; k < D * D; ++k) Gb[k] = 0.0;
#pragma unroll
    for (int cc = 0; cc < D; ++cc) nub += fb[cc] * lap[(int64_t)cc * n + o];
#pragma unroll
    for (int J2 = 0; J2 < D; ++J2) {
        double s = 0.0;
#pragma unroll
        for (int cc = 0; cc < D; ++cc) {
            Gb[cc * D + J2] += fb[cc] * gn[J2];
            Gb[J2 * D + cc] += fb[cc] * gn[J2];
            s += fb[cc] * (G[cc * D + J2] + G[J2 * D + cc]);
        }
        gnb[J2] = s;
    }
    double gnbh[D], b[D];
    jac_apply_t<D>(c.J[j], c.sx[j], c.sy[j], gnb, gnbh);
#pragma unroll
    for (int K = 0; K < D; ++K) {
        double s = 0.0;
#pragma unroll
        for (int L2 = 0; L2 < D; ++L2) s += W.L[(int64_t)(L2 * D + K) * cap + j] * gnbh[L2];
        b[K] = s;
    }
    // own share of the sum: -nu_j sum_k V_k grad w_jk . b
    double own = 0.0;
    for (int q = 0; q < cnt; ++q) {
        const int k = W.nbr[(int64_t)q * cap + j];
        if (c.type[k] == VIRTUAL) continue;
        double xk[3], r[D], rb = 0.0;
        load_hat<D>(c, k, xk);
#pragma unroll
        for (int K = 0; K < D; ++K) {
            r[K] = xk[K] - xj[K];
            rb += r[K] * b[K];
        }
        own += W.vol[k] * pair_fac<D>(P, r) * rb;
    }
    nub -= own;
#pragma unroll
    for (int K = 0; K < D; ++K) S[(int64_t)(RB + K) * cap + j] = b[K];
    S[(int64_t)RN * cap + j] = nub;
#pragma unroll
    for (int k = 0; k < D * D; ++k) S[(int64_t)(RG + k) * cap + j] = Gb[k];
}

// Eddy viscosity, second part, per particle k: nu_bar_k += sum over fluid j in S_k of
// V_k grad w_jk . b_j (its share of its neighbours' gn), then through
// nu_E = (C_s f_s r_e)^2 sqrt(2 S:S): G_bar += nu_bar nu_E S / (S:S), and
// grad^_bar = J^T G_bar per velocity component into the SPH(2) adjoint's gradient
// input (caller order, [(c d + K) n + orig]; 0 off the fluid).
template <int D>
__global__ void __launch_bounds__(128) k_stepadj_smag2(DevParams P, const Part c, Work W, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t cap = W.cap;
    const double *S = W.sadj;
    const int RB = 3 * D + D * D, RN = RB + D, RG = RN + 1;
    const int o = c.orig[k];
    double *gbar = W.sadj_co + (2 + 3 * D) * (int64_t)n;
    if (c.type[k] != FLUID) {
#pragma unroll
        for (int q = 0; q < D * D; ++q) gbar[(int64_t)q * n + o] = 0.0;
        return;
    }
    double xk[3], nub = S[(int64_t)RN * cap + k];
    load_hat<D>(c, k, xk);
    const double Vk = W.vol[k];
    const int cnt = W.nbr_cnt[k];
    for (int q = 0; q < cnt; ++q) {
        const int j = W.nbr[(int64_t)q * cap + k];
        if (c.type[j] != FLUID) continue;
        double xj[3], r[D], rb = 0.0;
        load_hat<D>(c, j, xj);
#pragma unroll
        for (int K = 0; K < D; ++K) {
            r[K] = xk[K] - xj[K];   // r_jk, seen from j
            rb += r[K] * S[(int64_t)(RB + K) * cap + j];
        }
        nub += Vk * pair_fac<D>(P, r) * rb;
    }
    double G[D * D], Gb[D * D], SS = 0.0, Sm[D * D];
#pragma unroll
    for (int cc = 0; cc < D; ++cc) {
        double gh[D], g[D];
#pragma unroll
        for (int K = 0; K < D; ++K) gh[K] = W.gv[(int64_t)(cc * D + K) * cap + k];
        jac_apply<D>(c.J[k], c.sx[k], c.sy[k], gh, g);
#pragma unroll
        for (int I = 0; I < D; ++I) G[I * D + cc] = g[I];
    }
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) {
            Sm[a * D + b] = 0.5 * (G[a * D + b] + G[b * D + a]);
            SS += Sm[a * D + b] * Sm[a * D + b];
        }
    const double nue = W.nu[k] - P.nu_k;
    const double s = SS > 0.0 ? nub * nue / SS : 0.0;
#pragma unroll
    for (int q = 0; q < D * D; ++q) Gb[q] = S[(int64_t)(RG + q) * cap + k] + s * Sm[q];
    // G[I d + c] = sum_K J[I][K] grad^[c d + K]: grad^_bar[c d + K] = (J^T G_bar[., c])_K
#pragma unroll
    for (int cc = 0; cc < D; ++cc) {
        double col[D], gh[D];
#pragma unroll
        for (int I = 0; I < D; ++I) col[I] = Gb[I * D + cc];
        jac_apply_t<D>(c.J[k], c.sx[k], c.sy[k], col, gh);
#pragma unroll
        for (int K = 0; K < D; ++K) gbar[(int64_t)(cc * D + K) * n + o] = gh[K];
    }
}

// Free-slip walls: wall j carries v_j = R_j sum_k V_k w_jk v_k / den_j (R_j = I - 2 n n^T,
// the Shepard average of its fluid neighbours reflected at the wall).  Its adjoint
// t_j (the viscous operator's phi_bar, in v_bar_in, plus the right side's, in W.sadj)
// becomes y_j = R_j t_j / den_j (rows [3d, 4d) of W.sadj, free on wall particles);
// k_stepadj_out hands V_k w_jk y_j to each fluid neighbour k.
template <int D>
__global__ void __launch_bounds__(128) k_stepadj_wall(DevParams P, const Part c, Work W, int n,
                                                      const double *v_bar_in)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n || c.type[j] != WALL) return;
    const int64_t cap = W.cap;
    const int o = c.orig[j];
    double xj[3], den = 0.0, nh[3] = {0.0, 0.0, 0.0};
    load_hat<D>(c, j, xj);
    const int cnt = W.nbr_cnt[j];
    for (int q = 0; q < cnt; ++q) {
        const int k = W.nbr[(int64_t)q * cap + j];
        const int tk = c.type[k];
        if (tk == WALL) continue;
        double xk[3], r[3], rr2 = 0.0;
        load_hat<D>(c, k, xk);
#pragma unroll
        for (int K = 0; K < D; ++K) {
            r[K] = xk[K] - xj[K];
            rr2 += r[K] * r[K];
        }
        const double rr = sqrt(rr2);
        double w, dw;
        kern_wdw<double>(rr, P.inv_l, P.ad, w, dw);
        if (tk == FLUID) den += W.vol[k] * w;
        else if (rr > 0.0) {
#pragma unroll
            for (int K = 0; K < D; ++K) nh[K] += P.V0 * (-dw / rr) * r[K];
        }
    }
    double y[D];
#pragma unroll
    for (int cc = 0; cc < D; ++cc) y[cc] = 0.0;
    if (den > 0.0) {
        double nn[D], nl = 0.0, tn = 0.0;
#pragma unroll
        for (int cc = 0; cc < D; ++cc)
            y[cc] = v_bar_in[(int64_t)cc * n + o] + W.sadj[(int64_t)(D + cc) * cap + j];
        jac_apply<D>(c.J[j], c.sx[j], c.sy[j], nh, nn);
#pragma unroll
        for (int I = 0; I < D; ++I) nl += nn[I] * nn[I];
        nl = sqrt(nl);
        if (nl > 0.0) {
#pragma unroll
            for (int I = 0; I < D; ++I) {
                nn[I] /= nl;
                tn += nn[I] * y[I];
            }
#pragma unroll
            for (int cc = 0; cc < D; ++cc) y[cc] -= 2.0 * tn * nn[cc];
        }
#pragma unroll
        for (int cc = 0; cc < D; ++cc) y[cc] /= den;
    }
#pragma unroll
    for (int cc = 0; cc < D; ++cc) W.sadj[(int64_t)(3 * D + cc) * cap + j] = y[cc];
}

// v_bar_in (holding the viscous term's phi_bar) += v*_bar on fluid particles, and
// with free-slip walls the wall neighbours' V_k w_jk y_j; 0 elsewhere.
template <int D>
__global__ void k_stepadj_out(DevParams P, const Part c, Work W, int n, double *v_bar_in)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t cap = W.cap;
    const int o = c.orig[i];
    if (c.type[i] != FLUID) {
#pragma unroll
        for (int cc = 0; cc < D; ++cc) v_bar_in[(int64_t)cc * n + o] = 0.0;
        return;
    }
    double t[D];
#pragma unroll
    for (int cc = 0; cc < D; ++cc)
        t[cc] = v_bar_in[(int64_t)cc * n + o] + W.sadj[(int64_t)(D + cc) * cap + i];
    if (P.slip) {
        double xi[3];
        load_hat<D>(c, i, xi);
        const double Vi = W.vol[i];
        const int cnt = W.nbr_cnt[i];
        for (int q = 0; q < cnt; ++q) {
            const int j = W.nbr[(int64_t)q * cap + i];
            if (c.type[j] != WALL) continue;
            double xj[3], rr2 = 0.0;
            load_hat<D>(c, j, xj);
#pragma unroll
            for (int K = 0; K < D; ++K) rr2 += (xi[K] - xj[K]) * (xi[K] - xj[K]);
            double w, dw;
            kern_wdw<double>(sqrt(rr2), P.inv_l, P.ad, w, dw);
#pragma unroll
            for (int cc = 0; cc < D; ++cc) t[cc] += Vi * w * W.sadj[(int64_t)(3 * D + cc) * cap + j];
        }
    }
#pragma unroll
    for (int cc = 0; cc < D; ++cc) v_bar_in[(int64_t)cc * n + o] = t[cc];
}

void launch_stepadj_a(const DevParams &P, Part cur, Work W, int64_t n, const double *v_bar,
                      const double *x_bar, const double *p_bar, cudaStream_t st)
{
    const unsigned g = (unsigned)((n + 127) / 128);
    const int D = P.dim;
    const bool sum = P.operators == 1;
    if (D == 2) {
        if (sum) {
            k_stepadj_corr<2, true><<<g, 128, 0, st>>>(P, cur, W, (int)n, v_bar, x_bar);
            k_stepadj_pbar<2, true><<<g, 128, 0, st>>>(P, cur, W, (int)n, p_bar);
        } else {
            k_stepadj_corr<2, false><<<g, 128, 0, st>>>(P, cur, W, (int)n, v_bar, x_bar);
            k_stepadj_pbar<2, false><<<g, 128, 0, st>>>(P, cur, W, (int)n, p_bar);
        }
        if (P.smag) k_stepadj_vcopy<2><<<g, 128, 0, st>>>(cur, W, (int)n);
    } else {
        if (sum) {
            k_stepadj_corr<3, true><<<g, 128, 0, st>>>(P, cur, W, (int)n, v_bar, x_bar);
            k_stepadj_pbar<3, true><<<g, 128, 0, st>>>(P, cur, W, (int)n, p_bar);
        } else {
            k_stepadj_corr<3, false><<<g, 128, 0, st>>>(P, cur, W, (int)n, v_bar, x_bar);
            k_stepadj_pbar<3, false><<<g, 128, 0, st>>>(P, cur, W, (int)n, p_bar);
        }
        if (P.smag) k_stepadj_vcopy<3><<<g, 128, 0, st>>>(cur, W, (int)n);
    }
    if (P.smag)   // the forward viscous term's Laplacian, for nu_bar
        launch_sph2_field(P, cur, W, n, W.sadj_co + (2 + D) * n, D, nullptr, nullptr,
                          W.sadj_co + (2 + 2 * D) * n, st);
}

void launch_stepadj_b(const DevParams &P, Part cur, Work W, int64_t n, cudaStream_t st)
{
    const unsigned g = (unsigned)((n + 127) / 128);
    if (P.dim == 2) {
        k_stepadj_rhs<2><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        k_stepadj_gather<2><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        if (P.smag) {
            k_stepadj_smag1<2><<<g, 128, 0, st>>>(P, cur, W, (int)n);
            k_stepadj_smag2<2><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        }
    } else {
        k_stepadj_rhs<3><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        k_stepadj_gather<3><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        if (P.smag) {
            k_stepadj_smag1<3><<<g, 128, 0, st>>>(P, cur, W, (int)n);
            k_stepadj_smag2<3><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        }
    }
}

void launch_stepadj_c(const DevParams &P, Part cur, Work W, int64_t n, double *v_bar_in,
                      cudaStream_t st)
{
    const unsigned g = (unsigned)((n + 127) / 128);
    if (P.dim == 2) {
        if (P.slip) k_stepadj_wall<2><<<g, 128, 0, st>>>(P, cur, W, (int)n, v_bar_in);
        k_stepadj_out<2><<<g, 128, 0, st>>>(P, cur, W, (int)n, v_bar_in);
    } else {
        if (P.slip) k_stepadj_wall<3><<<g, 128, 0, st>>>(P, cur, W, (int)n, v_bar_in);
        k_stepadj_out<3><<<g, 128, 0, st>>>(P, cur, W, (int)n, v_bar_in);
    }
}

// ---------------------------------------------------------------------------
// a12 (part): reverse of the particle regularisation (Sec. 4.1: dynamic
// stabilization, XSPH on free-surface particles, optimized shifting) at the
// positions x' and velocities u' the corrector left, for the step's reverse.
// Forward, per fluid particle i, with e_ij = r^'_j - r^'_i over the step's
// neighbour lists and free-surface flags:
//   du_i = -sum_j f_j (d_s - r)/(dt r) e_ij  (r < d_s = (1 - overlap) d0; f_j = 1/2 on fluid j)
//   ud_i = u'_i + T_i du_i,   dh_i = dt du_i        (T_i: projected to physical at x')
//   un_i = ud_i + eps sum_fluid j V0 (ud_j - ud_i) w_ij          (free-surface i only)
//   gc_i = sum_j V0 (w'/r)(-e_ij),  B_i = -sum_j V0 (w'/r) e_ij e_ij^T
//   s_i  = -K |v^_i| gc_i (K = shift l dt; v^ = the projected un), minus its part along
//          n_i = normalize(-B_i^-1 gc_i) on free-surface i
//   x''_i = x'_i + T_i (dh_i + s_i),   u''_i = un_i
// Its adjoint runs backwards through these lines: k_regadj_seed forms each
// particle's seeds (s's, v^'s and T's adjoints), k_regadj_vel the velocity
// adjoints (XSPH's transpose as a gather, du's), k_regadj_pos the pair terms'
// position adjoint (gathered from both ends of every pair, w' and w'' of the
// kernel) and k_regadj_out maps it to physical positions through the metric at
// x' (duals) and writes u'_bar and x'_bar (caller order) for the step's reverse.
// W.radj rows (cell order): gc_bar [0, d), B_bar [d, d + d^2), un_bar, h_bar
// (the projected displacement's adjoint), the metric's (J, s_x, s_y), x''_bar,
// du_bar, u'_bar, r^'_bar, x' (d rows each but the metric's 3).
// ---------------------------------------------------------------------------
template <int D>
struct RegRows {
    static constexpr int GC = 0, B = D, UN = D + D * D, H = 2 * D + D * D, M = 3 * D + D * D,
                         XD = M + 3, DU = XD + D, UP = DU + D, XH = UP + D, XP = XH + D,
                         N = XP + D;
};

// y = T^T x for T the projected-to-physical map of reg_to_phys; tb += the adjoint of
// T's entries (J, s_x, s_y) for the forward input dh and output dp.
template <int D>
__device__ __forceinline__ void reg_to_phys_t(double J, double sx, double sy, const double *dh,
                                              const double *xb, double *y, double *mb)
{
    if (D == 2) {
        const double dp1 = (dh[1] - sx * dh[0]) / J;
        y[0] = xb[0] - sx * xb[1] / J;
        y[1] = xb[1] / J;
        mb[0] += -xb[1] * dp1 / J;
        mb[1] += -xb[1] * dh[0] / J;
    } else {
        const double dp2 = (dh[2] - sx * dh[0] - sy * dh[1]) / J;
        y[0] = xb[0] - sx * xb[2] / J;
        y[1] = xb[1] - sy * xb[2] / J;
        y[2] = xb[2] / J;
        mb[0] += -xb[2] * dp2 / J;
        mb[1] += -xb[2] * dh[0] / J;
        mb[2] += -xb[2] * dh[1] / J;
    }
}

// x' (physical) before the regularisation moves it.
template <int D>
__global__ void k_regadj_save(const Part c, Work W, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    using RR = RegRows<D>;
    double x[3];
    load_phys<D>(c, i, x);
#pragma unroll
    for (int K = 0; K < D; ++K) W.radj[(int64_t)(RR::XP + K) * W.cap + i] = x[K];
}

template <int D>
__global__ void __launch_bounds__(128) k_regadj_seed(DevParams P, const Part c, Work W, int n,
                                                     const double *v_bar, const double *x_bar)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    using RR = RegRows<D>;
    const int64_t cap = W.cap;
    double *R = W.radj;
    if (c.type[i] != FLUID) {
        for (int q = 0; q < RR::XP; ++q) R[(int64_t)q * cap + i] = 0.0;
        return;
    }
    const int o = c.orig[i];
    const double J = W.rmet[i], sx = W.rmet[cap + i], sy = W.rmet[2 * cap + i];
    double xb[D], ub[D], un[D], rdh[D];
    load_vel<D>(c, i, un);   // the regularised velocity (the step's output)
#pragma unroll
    for (int K = 0; K < D; ++K) {
        xb[K] = x_bar ? x_bar[(int64_t)K * n + o] : 0.0;
        ub[K] = v_bar ? v_bar[(int64_t)K * n + o] : 0.0;
        rdh[K] = W.rdh[K * cap + i];
    }
    // forward shift (gc, B, s) at x'
    const bool fsi = W.fs[i] != 0, do_s = P.ops_shift > 0.0;
    double gc[D], B[D * D], s[D], sraw[D], nv[D], nn = 0.0, Df = 0.0, sp = 0.0, vh[D];
    bool proj = false;
#pragma unroll
    for (int K = 0; K < D; ++K) gc[K] = s[K] = sraw[K] = nv[K] = 0.0;
#pragma unroll
    for (int q = 0; q < D * D; ++q) B[q] = 0.0;
    if (do_s) {
        double xi[D];
#pragma unroll
        for (int K = 0; K < D; ++K) xi[K] = W.rxh[K * cap + i];
        const int cnt = W.nbr_cnt[i];
        for (int k = 0; k < cnt; ++k) {
            const int j = W.nbr[(int64_t)k * cap + i];
            double r[D], r2 = 0.0;
#pragma unroll
            for (int K = 0; K < D; ++K) {
                r[K] = xi[K] - W.rxh[K * cap + j];
                r2 += r[K] * r[K];
            }
            const double rr = sqrt(r2);
            if (rr == 0.0) continue;
            double w, dw;
            kern_wdw<double>(rr, P.inv_l, P.ad, w, dw);
            const double dwr = dw / rr;
#pragma unroll
            for (int K = 0; K < D; ++K) gc[K] += P.V0 * dwr * r[K];
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
                for (int b = 0; b < D; ++b) B[a * D + b] -= P.V0 * dwr * r[a] * r[b];
        }
        vh[0] = un[0];
        if (D == 2) {
            vh[1] = sx * un[0] + J * un[1];
        } else {
            vh[1] = un[1];
            vh[2] = sx * un[0] + sy * un[1] + J * un[2];
        }
#pragma unroll
        for (int K = 0; K < D; ++K) sp += vh[K] * vh[K];
        Df = P.ops_shift * P.l * sqrt(sp) * P.dt;
#pragma unroll
        for (int K = 0; K < D; ++K) s[K] = sraw[K] = -Df * gc[K];
        if (fsi) {
            double Bc[D * D], Li[D * D];
#pragma unroll
            for (int q = 0; q < D * D; ++q) Bc[q] = B[q];
            const bool ok = reg_invert<D>(Bc, Li);
            if (ok) {
#pragma unroll
                for (int a = 0; a < D; ++a) {
#pragma unroll
                    for (int b = 0; b < D; ++b) nv[a] -= Li[a * D + b] * gc[b];
                    nn += nv[a] * nv[a];
                }
            }
            if (!ok || !(nn > 0.0)) {
#pragma unroll
                for (int K = 0; K < D; ++K) s[K] = 0.0;
            } else {
                proj = true;
                nn = sqrt(nn);
                double sn = 0.0;
#pragma unroll
                for (int K = 0; K < D; ++K) sn += s[K] * nv[K] / nn;
#pragma unroll
                for (int K = 0; K < D; ++K) s[K] -= sn * nv[K] / nn;
            }
        }
    }
    // x'' = x' + T (dh + s)
    double dht[D], hb[D], mb[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int K = 0; K < D; ++K) dht[K] = rdh[K] + s[K];
    reg_to_phys_t<D>(J, sx, sy, dht, xb, hb, mb);
    double gcb[D], Bb[D * D], unb[D];
#pragma unroll
    for (int K = 0; K < D; ++K) {
        gcb[K] = 0.0;
        unb[K] = ub[K];
    }
#pragma unroll
    for (int q = 0; q < D * D; ++q) Bb[q] = 0.0;
    if (do_s && !(fsi && !proj)) {
        double srb[D];
        if (proj) {
            double n1[D], hn = 0.0, sn = 0.0, nb[D], nbn = 0.0;
#pragma unroll
            for (int K = 0; K < D; ++K) {
                n1[K] = nv[K] / nn;
                hn += hb[K] * n1[K];
                sn += sraw[K] * n1[K];
            }
#pragma unroll
            for (int K = 0; K < D; ++K) {
                srb[K] = hb[K] - hn * n1[K];
                nb[K] = -sn * hb[K] - hn * sraw[K];
                nbn += nb[K] * n1[K];
            }
            // n = nv / |nv|, nv = -B^-1 gc: nv_bar = (nb - (nb . n) n) / |nv|, y = B^-T nv_bar
            double nvb[D], Bt[D * D], Lt[D * D];
#pragma unroll
            for (int K = 0; K < D; ++K) nvb[K] = (nb[K] - nbn * n1[K]) / nn;
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
                for (int b = 0; b < D; ++b) Bt[a * D + b] = B[b * D + a];
            if (reg_invert<D>(Bt, Lt)) {
                double y[D];
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    y[a] = 0.0;
#pragma unroll
                    for (int b = 0; b < D; ++b) y[a] += Lt[a * D + b] * nvb[b];
                }
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    gcb[a] -= y[a];
#pragma unroll
                    for (int b = 0; b < D; ++b) Bb[a * D + b] -= y[a] * nv[b];
                }
            }
        } else {
#pragma unroll
            for (int K = 0; K < D; ++K) srb[K] = hb[K];
        }
        // s_raw = -Df gc, Df = K |v^|
        double Dfb = 0.0;
#pragma unroll
        for (int K = 0; K < D; ++K) {
            Dfb -= srb[K] * gc[K];
            gcb[K] -= Df * srb[K];
        }
        if (sp > 0.0) {
            const double kf = Dfb * P.ops_shift * P.l * P.dt / sqrt(sp);
            double vb[D];
#pragma unroll
            for (int K = 0; K < D; ++K) vb[K] = kf * vh[K];
            if (D == 2) {
                unb[0] += vb[0] + sx * vb[1];
                unb[1] += J * vb[1];
                mb[0] += un[1] * vb[1];
                mb[1] += un[0] * vb[1];
            } else {
                unb[0] += vb[0] + sx * vb[2];
                unb[1] += vb[1] + sy * vb[2];
                unb[2] += J * vb[2];
                mb[0] += un[2] * vb[2];
                mb[1] += un[0] * vb[2];
                mb[2] += un[1] * vb[2];
            }
        }
    }
#pragma unroll
    for (int K = 0; K < D; ++K) {
        R[(int64_t)(RR::GC + K) * cap + i] = gcb[K];
        R[(int64_t)(RR::UN + K) * cap + i] = unb[K];
        R[(int64_t)(RR::H + K) * cap + i] = hb[K];
        R[(int64_t)(RR::XD + K) * cap + i] = xb[K];
    }
#pragma unroll
    for (int q = 0; q < D * D; ++q) R[(int64_t)(RR::B + q) * cap + i] = Bb[q];
#pragma unroll
    for (int q = 0; q < 3; ++q) R[(int64_t)(RR::M + q) * cap + i] = mb[q];
}

// Velocity adjoints: ud_bar (XSPH's transpose gathered from free-surface fluid
// neighbours), then u'_bar = ud_bar and du_bar = T^T ud_bar + dt h_bar.
template <int D>
__global__ void __launch_bounds__(128) k_regadj_vel(DevParams P, const Part c, Work W, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n || c.type[k] != FLUID) return;
    using RR = RegRows<D>;
    const int64_t cap = W.cap;
    double *R = W.radj;
    const bool do_x = P.xsph_eps > 0.0;
    double udb[D], xk[D], wsum = 0.0;
#pragma unroll
    for (int K = 0; K < D; ++K) {
        udb[K] = 0.0;
        xk[K] = W.rxh[K * cap + k];
    }
    if (do_x) {
        const int cnt = W.nbr_cnt[k];
        for (int q = 0; q < cnt; ++q) {
            const int j = W.nbr[(int64_t)q * cap + k];
            if (c.type[j] != FLUID) continue;
            double r2 = 0.0;
#pragma unroll
            for (int K = 0; K < D; ++K) {
                const double dr = xk[K] - W.rxh[K * cap + j];
                r2 += dr * dr;
            }
            const double rr = sqrt(r2);
            if (rr == 0.0) continue;
            double w, dw;
            kern_wdw<double>(rr, P.inv_l, P.ad, w, dw);
            wsum += P.V0 * w;
            if (W.fs[j] != 0) {   // j's XSPH reads ud_k
#pragma unroll
                for (int K = 0; K < D; ++K) udb[K] += P.xsph_eps * P.V0 * w * R[(int64_t)(RR::UN + K) * cap + j];
            }
        }
    }
    const double own = (do_x && W.fs[k] != 0) ? 1.0 - P.xsph_eps * wsum : 1.0;
#pragma unroll
    for (int K = 0; K < D; ++K) udb[K] += own * R[(int64_t)(RR::UN + K) * cap + k];
    // ud = u' + T du (dynamic stabilization), dh = dt du
    const double J = W.rmet[k], sx = W.rmet[cap + k], sy = W.rmet[2 * cap + k];
    double du[D], dub[D], mb[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int K = 0; K < D; ++K) du[K] = W.rdh[K * cap + k] / P.dt;
    reg_to_phys_t<D>(J, sx, sy, du, udb, dub, mb);
#pragma unroll
    for (int K = 0; K < D; ++K) {
        R[(int64_t)(RR::UP + K) * cap + k] = udb[K];
        R[(int64_t)(RR::DU + K) * cap + k] = P.ds_overlap > 0.0 ? dub[K] + P.dt * R[(int64_t)(RR::H + K) * cap + k] : 0.0;
    }
    if (P.ds_overlap > 0.0)
#pragma unroll
        for (int q = 0; q < 3; ++q) R[(int64_t)(RR::M + q) * cap + k] += mb[q];
}

// Adjoint of pair (i, j)'s terms owned by fluid particle i with respect to its
// separation e = r^'_j - r^'_i.  T: the pair arithmetic's type (the mixed form's
// FP32, as its forward regularisation's pair sums; the separation itself is
// formed in FP64 first), one reciprocal of |e| per pair.
template <int D, typename T>
__device__ __forceinline__ void reg_pair_ebar(const DevParams &P, const Part &c, const Work &W, int i,
                                              int j, T *eb)
{
    using RR = RegRows<D>;
    const int64_t cap = W.cap;
    const double *R = W.radj;
    T e[D], r2 = T(0);
#pragma unroll
    for (int K = 0; K < D; ++K) {
        e[K] = (T)(W.rxh[K * cap + j] - W.rxh[K * cap + i]);
        r2 += e[K] * e[K];
        eb[K] = T(0);
    }
    if (r2 == T(0)) return;
    const T rr = sqrt(r2), ir = T(1) / rr;
    const int tj = c.type[j];
    const T dds = (T)((1.0 - P.ds_overlap) * P.d0);
    if (P.ds_overlap > 0.0 && rr < dds) {
        const T idt = (T)(1.0 / P.dt), f = tj == FLUID ? T(0.5) : T(1);
        const T g = (dds - rr) * idt * ir, gp = -dds * idt * ir * ir;
        T du[D], de = T(0);
#pragma unroll
        for (int K = 0; K < D; ++K) {
            du[K] = (T)R[(int64_t)(RR::DU + K) * cap + i];
            de += du[K] * e[K];
        }
#pragma unroll
        for (int K = 0; K < D; ++K) eb[K] -= f * (g * du[K] + de * gp * e[K] * ir);
    }
    T w, dw;
    kern_wdw<T>(rr, (T)P.inv_l, (T)P.ad, w, dw);
    if (P.xsph_eps > 0.0 && W.fs[i] != 0 && tj == FLUID) {
        T sdot = T(0);
#pragma unroll
        for (int K = 0; K < D; ++K)
            sdot += (T)R[(int64_t)(RR::UN + K) * cap + i] * (T)(W.rud[K * cap + j] - W.rud[K * cap + i]);
        const T fx = (T)(P.xsph_eps * P.V0) * sdot * dw * ir;
#pragma unroll
        for (int K = 0; K < D; ++K) eb[K] += fx * e[K];
    }
    if (P.ops_shift > 0.0) {   // forward separation r_s = -e
        const T phi = dw * ir, dphi = (kern_w2t<T>(rr, (T)P.inv_l, (T)P.ad) - phi) * ir;
        T gb[D], Bb[D * D], rs[D], gr = T(0), rBr = T(0), Brs[D];
#pragma unroll
        for (int K = 0; K < D; ++K) {
            gb[K] = (T)R[(int64_t)(RR::GC + K) * cap + i];
            rs[K] = -e[K];
            gr += gb[K] * rs[K];
        }
#pragma unroll
        for (int q = 0; q < D * D; ++q) Bb[q] = (T)R[(int64_t)(RR::B + q) * cap + i];
#pragma unroll
        for (int a2 = 0; a2 < D; ++a2) {
            Brs[a2] = T(0);
#pragma unroll
            for (int b2 = 0; b2 < D; ++b2) Brs[a2] += (Bb[a2 * D + b2] + Bb[b2 * D + a2]) * rs[b2];
#pragma unroll
            for (int b2 = 0; b2 < D; ++b2) rBr += rs[a2] * Bb[a2 * D + b2] * rs[b2];
        }
        const T V0 = (T)P.V0, sc = (gr - rBr) * dphi * ir;
#pragma unroll
        for (int K = 0; K < D; ++K)
            eb[K] -= V0 * (phi * (gb[K] - Brs[K]) + sc * rs[K]);   // d/de = -d/dr_s
    }
}

template <int D, typename T>
__global__ void __launch_bounds__(128) k_regadj_pos(DevParams P, const Part c, Work W, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n || c.type[k] != FLUID) return;
    using RR = RegRows<D>;
    const int64_t cap = W.cap;
    double rb[D];
    T eb[D];
#pragma unroll
    for (int K = 0; K < D; ++K) rb[K] = 0.0;
    const int cnt = W.nbr_cnt[k];
    for (int q = 0; q < cnt; ++q) {
        const int j = W.nbr[(int64_t)q * cap + k];
        reg_pair_ebar<D, T>(P, c, W, k, j, eb);   // k's own pair: e = r^_j - r^_k
#pragma unroll
        for (int K = 0; K < D; ++K) rb[K] -= (double)eb[K];
        if (c.type[j] == FLUID) {
            reg_pair_ebar<D, T>(P, c, W, j, k, eb);   // j's pair: e = r^_k - r^_j
#pragma unroll
            for (int K = 0; K < D; ++K) rb[K] += (double)eb[K];
        }
    }
#pragma unroll
    for (int K = 0; K < D; ++K) W.radj[(int64_t)(RR::XH + K) * cap + k] = rb[K];
}

// Physical x'_bar = (d r^'/d x')^T r^'_bar + the metric's adjoint through duals at x'
// + x''_bar; writes u'_bar and x'_bar in caller order (0 off the fluid).
template <int D>
__global__ void __launch_bounds__(128) k_regadj_out(DevParams P, const Part c, Work W, int n,
                                                    double *vb_co, double *xb_co)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    using RR = RegRows<D>;
    const int64_t cap = W.cap;
    const double *R = W.radj;
    const int o = c.orig[k];
    if (c.type[k] != FLUID) {
#pragma unroll
        for (int K = 0; K < D; ++K) vb_co[(int64_t)K * n + o] = xb_co[(int64_t)K * n + o] = 0.0;
        return;
    }
    const double J = W.rmet[k], sx = W.rmet[cap + k], sy = W.rmet[2 * cap + k];
    double a[D], xb[D], xp[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int K = 0; K < D; ++K) {
        a[K] = R[(int64_t)(RR::XH + K) * cap + k];
        xp[K] = R[(int64_t)(RR::XP + K) * cap + k];
    }
    // r^ = (x, [y], z^(x, y, z)): d z^/d(x, y, z) = (s_x, s_y, J)
    xb[0] = a[0] + sx * a[D - 1];
    if (D == 3) xb[1] = a[1] + sy * a[2];
    xb[D - 1] = J * a[D - 1];
    const double mJ = R[(int64_t)RR::M * cap + k], msx = R[(int64_t)(RR::M + 1) * cap + k],
                 msy = R[(int64_t)(RR::M + 2) * cap + k];
    const double x = xp[0], y = D == 3 ? xp[1] : 0.0, z = xp[D - 1];
    for (int K = 0; K < D; ++K) {
        const int axis = D == 3 ? K : (K == 0 ? 0 : 2);
        Dual out[6];
        metric_dual(P, Dual(x, axis == 0 ? 1.0 : 0.0), Dual(y, axis == 1 ? 1.0 : 0.0),
                    Dual(z, axis == 2 ? 1.0 : 0.0), -1, out);
        xb[K] += mJ * out[1].d + msx * out[2].d + msy * out[3].d;
    }
#pragma unroll
    for (int K = 0; K < D; ++K) {
        vb_co[(int64_t)K * n + o] = R[(int64_t)(RR::UP + K) * cap + k];
        xb_co[(int64_t)K * n + o] = xb[K] + R[(int64_t)(RR::XD + K) * cap + k];
    }
}

int regadj_rows(int dim) { return dim == 2 ? RegRows<2>::N : RegRows<3>::N; }

void launch_regadj_save(const DevParams &P, Part cur, Work W, int64_t n, cudaStream_t st)
{
    const unsigned g = (unsigned)((n + 127) / 128);
    if (P.dim == 2) k_regadj_save<2><<<g, 128, 0, st>>>(cur, W, (int)n);
    else k_regadj_save<3><<<g, 128, 0, st>>>(cur, W, (int)n);
}

void launch_regadj(const DevParams &P, Part cur, Work W, int64_t n, const double *v_bar,
                   const double *x_bar, double *vb_co, double *xb_co, cudaStream_t st)
{
    const unsigned g = (unsigned)((n + 127) / 128);
    if (P.dim == 2) {
        k_regadj_seed<2><<<g, 128, 0, st>>>(P, cur, W, (int)n, v_bar, x_bar);
        k_regadj_vel<2><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        if (P.precision == VCT_MIXED) k_regadj_pos<2, float><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        else k_regadj_pos<2, double><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        k_regadj_out<2><<<g, 128, 0, st>>>(P, cur, W, (int)n, vb_co, xb_co);
    } else {
        k_regadj_seed<3><<<g, 128, 0, st>>>(P, cur, W, (int)n, v_bar, x_bar);
        k_regadj_vel<3><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        if (P.precision == VCT_MIXED) k_regadj_pos<3, float><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        else k_regadj_pos<3, double><<<g, 128, 0, st>>>(P, cur, W, (int)n);
        k_regadj_out<3><<<g, 128, 0, st>>>(P, cur, W, (int)n, vb_co, xb_co);
    }
}


// ---------------------------------------------------------------------------
// a12 (part): derivative of the corrected gradient <grad^ phi>_i = L_i g_i,
// g_i = sum_j V_j (phi_j - phi_i) grad w_ij, L_i = B_i^-1, B_i = sum_j V_j
// grad w_ij (x) r_ij (Eq. gra_1st; fluid and wall neighbours), with respect to
// the projected positions, through w' and w'' of the kernel; neighbour sets and
// volumes held fixed.  With grad w_ij = f(rho) r_ij, f = -w'/rho, rho = |r_ij|,
// r_ij = r_j - r_i, its Jacobian is H = f I + (f'/rho) r r^T, f' = (w' - w''
// rho) / rho^2.  For the loss sum_i Gbar_i . G_i: gbar_i = L_i^T Gbar_i,
// Bbar_i = -L_i^T (sum_c Gbar_i,c g_i,c^T) L_i^T (the inverse's adjoint), and
// pair (i, j) adds rbar_ij = V_j [H (sum_c dphi_c gbar_i,c + Bbar_i r) +
// Bbar_i^T f r] to r_j and subtracts it from r_i.  k_gradpos_a forms gbar_i
// and Bbar_i per fluid particle (into the pass-1 scratch W.Ct and W.gv);
// k_gradpos_b gathers every particle's sum over its pairs from both ends (the
// neighbour relation is symmetric), deterministic.  FP64.
// ---------------------------------------------------------------------------

template <int D>
__global__ void __launch_bounds__(128) k_gradpos_a(DevParams P, const Part c, Work W, int n,
                                                   int ncomp, const double *phi,
                                                   const double *grad_bar)
{
    if (step_failed(W.status)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || c.type[i] != FLUID) return;
    const int64_t cap = W.cap;
    double xi[3];
    load_hat<D>(c, i, xi);
    const int oi = c.orig[i];
    double B[D * D], g[3][D];
#pragma unroll
    for (int q = 0; q < D * D; ++q) B[q] = 0.0;
    for (int cc = 0; cc < 3; ++cc)
#pragma unroll
        for (int K = 0; K < D; ++K) g[cc][K] = 0.0;
    const int cnt = W.nbr_cnt[i];
    for (int k = 0; k < cnt; ++k) {
        const int j = W.nbr[(int64_t)k * cap + i];
        if (c.type[j] == VIRTUAL) continue;
        double xj[3], r[D], rr2 = 0.0;
        load_hat<D>(c, j, xj);
#pragma unroll
        for (int K = 0; K < D; ++K) {
            r[K] = xj[K] - xi[K];
            rr2 += r[K] * r[K];
        }
        if (rr2 == 0.0) continue;
        const double rr = sqrt(rr2);
        double w, dw;
        kern_wdw<double>(rr, P.inv_l, P.ad, w, dw);
        const double f = -dw / rr, V = W.vol[j];
#pragma unroll
        for (int K = 0; K < D; ++K)
#pragma unroll
            for (int L2 = 0; L2 < D; ++L2) B[K * D + L2] += V * f * r[K] * r[L2];
        const int oj = c.orig[j];
        for (int cc = 0; cc < ncomp; ++cc) {
            const double dphi = phi[(int64_t)cc * n + oj] - phi[(int64_t)cc * n + oi];
#pragma unroll
            for (int K = 0; K < D; ++K) g[cc][K] += V * dphi * f * r[K];
        }
    }
    double L[D * D];
    if (!inv_small<D>(B, L)) {
        set_error(W.status, VCT_ERR_SINGULAR, i);
        return;
    }
    double Lbar[D * D];
#pragma unroll
    for (int q = 0; q < D * D; ++q) Lbar[q] = 0.0;
    for (int cc = 0; cc < ncomp; ++cc) {
        double Gb[D];
#pragma unroll
        for (int K = 0; K < D; ++K) Gb[K] = grad_bar[((int64_t)cc * D + K) * n + oi];
#pragma unroll
        for (int K = 0; K < D; ++K) {   // gbar = L^T Gbar
            double s = 0.0;
#pragma unroll
            for (int M2 = 0; M2 < D; ++M2) s += L[M2 * D + K] * Gb[M2];
            W.Ct[((int64_t)cc * D + K) * cap + i] = s;
        }
#pragma unroll
        for (int K = 0; K < D; ++K)
#pragma unroll
            for (int L2 = 0; L2 < D; ++L2) Lbar[K * D + L2] += Gb[K] * g[cc][L2];
    }
    // Bbar = -L^T Lbar L^T
    double T[D * D];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) {
            double s = 0.0;
#pragma unroll
            for (int m = 0; m < D; ++m) s += L[m * D + a] * Lbar[m * D + b];
            T[a * D + b] = s;
        }
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) {
            double s = 0.0;
#pragma unroll
            for (int m = 0; m < D; ++m) s += T[a * D + m] * L[b * D + m];
            W.gv[(int64_t)(a * D + b) * cap + i] = -s;
        }
}

// rbar of pair (i, j) at r = r_j - r_i, from i's gbar and Bbar
template <int D>
__device__ __forceinline__ void gradpos_pair(const Work &W, int i, int ncomp, const double *dphi,
                                             const double *r, double rr, double f, double fp,
                                             double V, double *rb)
{
    const int64_t cap = W.cap;
    double v[D], Bt[D];
#pragma unroll
    for (int K = 0; K < D; ++K) {
        double s = 0.0, t = 0.0;
        for (int cc = 0; cc < ncomp; ++cc) s += dphi[cc] * W.Ct[((int64_t)cc * D + K) * cap + i];
#pragma unroll
        for (int L2 = 0; L2 < D; ++L2) {
            s += W.gv[(int64_t)(K * D + L2) * cap + i] * r[L2];        // Bbar r
            t += W.gv[(int64_t)(L2 * D + K) * cap + i] * f * r[L2];    // Bbar^T f r
        }
        v[K] = s;
        Bt[K] = t;
    }
    double rv = 0.0;
#pragma unroll
    for (int K = 0; K < D; ++K) rv += r[K] * v[K];
#pragma unroll
    for (int K = 0; K < D; ++K) rb[K] = V * (f * v[K] + fp / rr * r[K] * rv + Bt[K]);
}

template <int D>
__global__ void __launch_bounds__(128) k_gradpos_b(DevParams P, const Part c, Work W, int n,
                                                   int ncomp, const double *phi, double *xh_bar)
{
    if (step_failed(W.status)) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t cap = W.cap;
    const int tk = c.type[k], ok = c.orig[k];
    double out[D];
#pragma unroll
    for (int K = 0; K < D; ++K) out[K] = 0.0;
    if (tk != VIRTUAL) {
        double xk[3];
        load_hat<D>(c, k, xk);
        const int cnt = W.nbr_cnt[k];
        for (int q = 0; q < cnt; ++q) {
            const int m = W.nbr[(int64_t)q * cap + k];
            const int tm = c.type[m];
            if (tm == VIRTUAL) continue;
            if (tk != FLUID && tm != FLUID) continue;
            double xm[3], r[D], rn[D], rr2 = 0.0;
            load_hat<D>(c, m, xm);
#pragma unroll
            for (int K = 0; K < D; ++K) {
                r[K] = xm[K] - xk[K];   // r_km
                rn[K] = -r[K];          // r_mk
                rr2 += r[K] * r[K];
            }
            if (rr2 == 0.0) continue;
            const double rr = sqrt(rr2);
            double w, dw;
            kern_wdw<double>(rr, P.inv_l, P.ad, w, dw);
            const double w2 = kern_w2(rr, P.inv_l, P.ad);
            const double f = -dw / rr, fp = (dw - w2 * rr) / (rr * rr);
            const int om = c.orig[m];
            double dphi[3], rb[D];
            if (tk == FLUID) {   // pair (k, m): rbar_km leaves r_k
                for (int cc = 0; cc < ncomp; ++cc)
                    dphi[cc] = phi[(int64_t)cc * n + om] - phi[(int64_t)cc * n + ok];
                gradpos_pair<D>(W, k, ncomp, dphi, r, rr, f, fp, W.vol[m], rb);
#pragma unroll
                for (int K = 0; K < D; ++K) out[K] -= rb[K];
            }
            if (tm == FLUID) {   // pair (m, k): rbar_mk arrives at r_k
                for (int cc = 0; cc < ncomp; ++cc)
                    dphi[cc] = phi[(int64_t)cc * n + ok] - phi[(int64_t)cc * n + om];
                gradpos_pair<D>(W, m, ncomp, dphi, rn, rr, f, fp, W.vol[k], rb);
#pragma unroll
                for (int K = 0; K < D; ++K) out[K] += rb[K];
            }
        }
    }
#pragma unroll
    for (int K = 0; K < D; ++K) xh_bar[(int64_t)K * n + ok] = out[K];
}

void launch_gradpos(const DevParams &P, Part cur, Work W, int64_t n, int ncomp, const double *phi,
                    const double *grad_bar, double *xh_bar, cudaStream_t st)
{
    const unsigned g = (unsigned)((n + 127) / 128);
    if (P.dim == 2) {
        k_gradpos_a<2><<<g, 128, 0, st>>>(P, cur, W, (int)n, ncomp, phi, grad_bar);
        k_gradpos_b<2><<<g, 128, 0, st>>>(P, cur, W, (int)n, ncomp, phi, xh_bar);
    } else {
        k_gradpos_a<3><<<g, 128, 0, st>>>(P, cur, W, (int)n, ncomp, phi, grad_bar);
        k_gradpos_b<3><<<g, 128, 0, st>>>(P, cur, W, (int)n, ncomp, phi, xh_bar);
    }
}


// ---------------------------------------------------------------------------
// a12 (part): derivative of the SPH(2) second derivatives (Eq. sec_SPH2,
// D = 2 M_i^-1 b_i, cross terms halved in the output) with respect to the
// projected positions, neighbour sets and volumes held fixed.  Per fluid
// particle i, with gt = L_i grad w, F = r.gt / rho^4, q = q(r), p = q - C_i^T r
// (C_i = L_i sum V grad w q^T), e = phi_ij - r.g_i (g_i the corrected
// gradient): M_i = sum V F q p^T, b_i = sum V F q e.  Reverse: xbar = 2 Dbar,
// bbar = M^-T xbar, Mbar = -bbar x^T; per pair Fbar = V (q.bbar)(e - x.p),
// qbar = V F (e - x.p) bbar + pbar, pbar = -V F (q.bbar) x, ebar = V F (q.bbar),
// which feed gbar = -sum ebar r, Cbar = -sum r pbar^T and Lbar (through gt),
// then Lbar += gbar g_raw^T + Cbar Gq^T, Bbar = -L^T Lbar L^T, and every term's
// dependence on r (through rho, grad w, q, p, e) gives the pair's rbar.
// k_d2pos_a forms and stores i's factors and adjoints (L, C, g, x, bbar,
// L^T gbar, L^T Cbar, Bbar: 2d^2 + 2dm + 2d + 2m doubles, in the scratch of the
// pressure-equation coefficients, which the next step rebuilds); k_d2pos_b
// gathers each particle's sum over its pairs from both ends.  FP64, one field.
// ---------------------------------------------------------------------------
template <int D>
struct D2Slots {
    static constexpr int M = D == 2 ? 3 : 6;
    static constexpr int L = 0, C = L + D * D, G = C + D * M, X = G + D, BB = X + M, GR = BB + M,
                         GQ = GR + D, BBAR = GQ + D * M, N = BBAR + D * D;
};

template <int D>
__device__ __forceinline__ void qvec_d(const double *r, double *q)
{
    if (D == 2) {
        q[0] = r[0] * r[0]; q[1] = r[1] * r[1]; q[2] = r[0] * r[1];
    } else {
        q[0] = r[0] * r[0]; q[1] = r[1] * r[1]; q[2] = r[2] * r[2];
        q[3] = r[0] * r[1]; q[4] = r[1] * r[2]; q[5] = r[2] * r[0];
    }
}

// (dq/dr)^T qb
template <int D>
__device__ __forceinline__ void qjac_t(const double *r, const double *qb, double *out)
{
    if (D == 2) {
        out[0] = 2.0 * r[0] * qb[0] + r[1] * qb[2];
        out[1] = 2.0 * r[1] * qb[1] + r[0] * qb[2];
    } else {
        out[0] = 2.0 * r[0] * qb[0] + r[1] * qb[3] + r[2] * qb[5];
        out[1] = 2.0 * r[1] * qb[1] + r[0] * qb[3] + r[2] * qb[4];
        out[2] = 2.0 * r[2] * qb[2] + r[1] * qb[4] + r[0] * qb[5];
    }
}

// PPE = false: a field phi, the loss sum d2_bar . d2_hat.  PPE = true: the
// pressure operator's linear part (A x)_i = c0_i <dx/dz^>_i + c~_i . D_i (Eqs.
// VCT_ppe, lap_VCT) on the unknown rows, with pair differences x_j - x_i for
// fluid neighbours (x = 0 off the unknowns) and none for walls (their term is
// the right side's), the loss sum_i pbar_i (A x)_i; phi = x, wbar = pbar.
template <int D>
__device__ __forceinline__ double d2pos_dphi(const Part &c, const Work &W, bool ppe,
                                             const double *phi, int i, int j)
{
    if (!ppe) return phi[c.orig[j]] - phi[c.orig[i]];
    if (c.type[j] != FLUID) return 0.0;
    const double xj = W.fs[j] ? 0.0 : phi[c.orig[j]];
    return xj - phi[c.orig[i]];
}

template <int D, bool PPE>
__global__ void __launch_bounds__(128) k_d2pos_a(DevParams P, const Part c, Work W, int n,
                                                 const double *phi, const double *wbar,
                                                 double *scr)
{
    constexpr int M = D2Slots<D>::M;
    using SL = D2Slots<D>;
    if (step_failed(W.status)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || c.type[i] != FLUID) return;
    const int64_t cap = W.cap;
    double xi[3];
    load_hat<D>(c, i, xi);
    const int oi = c.orig[i];
    double B[D * D], Gq[D * M], graw[D];
    for (int q = 0; q < D * D; ++q) B[q] = 0.0;
    for (int q = 0; q < D * M; ++q) Gq[q] = 0.0;
    for (int K = 0; K < D; ++K) graw[K] = 0.0;
    const int cnt = W.nbr_cnt[i];
    for (int k = 0; k < cnt; ++k) {   // B, Gq, g_raw
        const int j = W.nbr[(int64_t)k * cap + i];
        if (c.type[j] == VIRTUAL) continue;
        double xj[3], r[D], rr2 = 0.0, q[M];
        load_hat<D>(c, j, xj);
        for (int K = 0; K < D; ++K) { r[K] = xj[K] - xi[K]; rr2 += r[K] * r[K]; }
        if (rr2 == 0.0) continue;
        const double rr = sqrt(rr2);
        double w, dw;
        kern_wdw<double>(rr, P.inv_l, P.ad, w, dw);
        const double f = -dw / rr, V = W.vol[j], dphi = d2pos_dphi<D>(c, W, PPE, phi, i, j);
        qvec_d<D>(r, q);
        for (int K = 0; K < D; ++K) {
            const double gk = f * r[K];
            for (int L2 = 0; L2 < D; ++L2) B[K * D + L2] += V * gk * r[L2];
            for (int a = 0; a < M; ++a) Gq[K * M + a] += V * gk * q[a];
            graw[K] += V * dphi * gk;
        }
    }
    double L[D * D];
    if (!inv_small<D>(B, L)) {
        set_error(W.status, VCT_ERR_SINGULAR, i);
        return;
    }
    double C[D * M], g[D];
    for (int K = 0; K < D; ++K) {
        g[K] = 0.0;
        for (int L2 = 0; L2 < D; ++L2) g[K] += L[K * D + L2] * graw[L2];
        for (int a = 0; a < M; ++a) {
            double s2 = 0.0;
            for (int L2 = 0; L2 < D; ++L2) s2 += L[K * D + L2] * Gq[L2 * M + a];
            C[K * M + a] = s2;
        }
    }
    double Mm[M * M], b[M];
    for (int q = 0; q < M * M; ++q) Mm[q] = 0.0;
    for (int a = 0; a < M; ++a) b[a] = 0.0;
    for (int k = 0; k < cnt; ++k) {   // M, b
        const int j = W.nbr[(int64_t)k * cap + i];
        if (c.type[j] == VIRTUAL) continue;
        double xj[3], r[D], rr2 = 0.0, q[M], pv[M], gt[D];
        load_hat<D>(c, j, xj);
        for (int K = 0; K < D; ++K) { r[K] = xj[K] - xi[K]; rr2 += r[K] * r[K]; }
        if (rr2 == 0.0) continue;
        const double rr = sqrt(rr2);
        double w, dw;
        kern_wdw<double>(rr, P.inv_l, P.ad, w, dw);
        const double f = -dw / rr, V = W.vol[j], dphi = d2pos_dphi<D>(c, W, PPE, phi, i, j);
        double rg = 0.0, rgg = 0.0;
        for (int K = 0; K < D; ++K) {
            double s2 = 0.0;
            for (int L2 = 0; L2 < D; ++L2) s2 += L[K * D + L2] * f * r[L2];
            gt[K] = s2;
            rg += r[K] * s2;
            rgg += r[K] * g[K];
        }
        const double F = rg / (rr2 * rr2), e = dphi - rgg;
        qvec_d<D>(r, q);
        for (int a = 0; a < M; ++a) {
            double s2 = 0.0;
            for (int K = 0; K < D; ++K) s2 += C[K * M + a] * r[K];
            pv[a] = q[a] - s2;
        }
        for (int a = 0; a < M; ++a) {
            for (int bq = 0; bq < M; ++bq) Mm[a * M + bq] += V * F * q[a] * pv[bq];
            b[a] += V * F * q[a] * e;
        }
    }
    int piv[M];
    if (!lu_factor<M>(Mm, piv)) {
        set_error(W.status, VCT_ERR_SINGULAR, i);
        return;
    }
    double x[M], bb[M];
    for (int a = 0; a < M; ++a) x[a] = b[a];
    lu_apply<M, 1>(Mm, piv, x);
    double gdir[D];   // the loss's own weight on the corrected gradient
    for (int K = 0; K < D; ++K) gdir[K] = 0.0;
    if (PPE) {   // xbar = 2 pbar c~ on D; pbar c0 on the gradient's z^ component
        const double pb = W.fs[i] ? 0.0 : wbar[oi];
        double ct[M];
        ctilde<D>(c.c3[i], c.sx[i], c.sy[i], ct);
        for (int a = 0; a < M; ++a) bb[a] = 2.0 * pb * ct[a];
        gdir[D - 1] = pb * c.c0[i];
    } else {
        for (int a = 0; a < M; ++a) {   // xbar = 2 Dbar, the output's cross terms halved
            const double db = wbar[(int64_t)a * n + oi];
            bb[a] = 2.0 * (a < D ? db : 0.5 * db);
        }
    }
    lu_apply_t<M>(Mm, piv, bb);
    double gb[D], Cb[D * M], Lb[D * D];
    for (int K = 0; K < D; ++K) gb[K] = gdir[K];
    for (int q = 0; q < D * M; ++q) Cb[q] = 0.0;
    for (int q = 0; q < D * D; ++q) Lb[q] = 0.0;
    for (int k = 0; k < cnt; ++k) {   // per-i sums of the pair adjoints
        const int j = W.nbr[(int64_t)k * cap + i];
        if (c.type[j] == VIRTUAL) continue;
        double xj[3], r[D], rr2 = 0.0, q[M], pv[M], gw[D];
        load_hat<D>(c, j, xj);
        for (int K = 0; K < D; ++K) { r[K] = xj[K] - xi[K]; rr2 += r[K] * r[K]; }
        if (rr2 == 0.0) continue;
        const double rr = sqrt(rr2);
        double w, dw;
        kern_wdw<double>(rr, P.inv_l, P.ad, w, dw);
        const double f = -dw / rr, V = W.vol[j], dphi = d2pos_dphi<D>(c, W, PPE, phi, i, j);
        double rg = 0.0, rgg = 0.0;
        for (int K = 0; K < D; ++K) gw[K] = f * r[K];
        for (int K = 0; K < D; ++K) {
            double s2 = 0.0;
            for (int L2 = 0; L2 < D; ++L2) s2 += L[K * D + L2] * gw[L2];
            rg += r[K] * s2;
            rgg += r[K] * g[K];
        }
        const double F = rg / (rr2 * rr2), e = dphi - rgg;
        qvec_d<D>(r, q);
        double qbd = 0.0, xp = 0.0;
        for (int a = 0; a < M; ++a) {
            double s2 = 0.0;
            for (int K = 0; K < D; ++K) s2 += C[K * M + a] * r[K];
            pv[a] = q[a] - s2;
            qbd += q[a] * bb[a];
        }
        for (int a = 0; a < M; ++a) xp += x[a] * pv[a];
        const double Fb = V * qbd * (e - xp), eb = V * F * qbd;
        for (int K = 0; K < D; ++K) gb[K] -= eb * r[K];
        for (int K = 0; K < D; ++K)
            for (int a = 0; a < M; ++a) Cb[K * M + a] += r[K] * V * F * qbd * x[a];   // -r pbar^T
        const double rgb = Fb / (rr2 * rr2);
        for (int K = 0; K < D; ++K)
            for (int L2 = 0; L2 < D; ++L2) Lb[K * D + L2] += rgb * r[K] * gw[L2];
    }
    for (int K = 0; K < D; ++K)
        for (int L2 = 0; L2 < D; ++L2) {
            double s2 = gb[K] * graw[L2];
            for (int a = 0; a < M; ++a) s2 += Cb[K * M + a] * Gq[L2 * M + a];
            Lb[K * D + L2] += s2;
        }
    double gr[D], Gqb[D * M], T[D * D];
    for (int K = 0; K < D; ++K) {
        double s2 = 0.0;
        for (int L2 = 0; L2 < D; ++L2) s2 += L[L2 * D + K] * gb[L2];
        gr[K] = s2;
        for (int a = 0; a < M; ++a) {
            double s3 = 0.0;
            for (int L2 = 0; L2 < D; ++L2) s3 += L[L2 * D + K] * Cb[L2 * M + a];
            Gqb[K * M + a] = s3;
        }
    }
    for (int a = 0; a < D; ++a)
        for (int bq = 0; bq < D; ++bq) {
            double s2 = 0.0;
            for (int m2 = 0; m2 < D; ++m2) s2 += L[m2 * D + a] * Lb[m2 * D + bq];
            T[a * D + bq] = s2;
        }
    auto st = [&](int slot, double v) { scr[(int64_t)slot * cap + i] = v; };
    for (int q = 0; q < D * D; ++q) st(SL::L + q, L[q]);
    for (int q = 0; q < D * M; ++q) st(SL::C + q, C[q]);
    for (int K = 0; K < D; ++K) st(SL::G + K, g[K]);
    for (int a = 0; a < M; ++a) st(SL::X + a, x[a]);
    for (int a = 0; a < M; ++a) st(SL::BB + a, bb[a]);
    for (int K = 0; K < D; ++K) st(SL::GR + K, gr[K]);
    for (int q = 0; q < D * M; ++q) st(SL::GQ + q, Gqb[q]);
    for (int a = 0; a < D; ++a)
        for (int bq = 0; bq < D; ++bq) {
            double s2 = 0.0;
            for (int m2 = 0; m2 < D; ++m2) s2 += T[a * D + m2] * L[bq * D + m2];
            st(SL::BBAR + a * D + bq, -s2);
        }
}

// rbar of pair (i, j) at r = r_j - r_i from i's stored factors and adjoints
template <int D>
__device__ void d2pos_pair(const DevParams &P, const double *scr, int64_t cap, int i, double dphi,
                           const double *r, double V, double *rb)
{
    constexpr int M = D2Slots<D>::M;
    using SL = D2Slots<D>;
    auto ld = [&](int slot) { return scr[(int64_t)slot * cap + i]; };
    double rr2 = 0.0;
    for (int K = 0; K < D; ++K) rr2 += r[K] * r[K];
    const double rr = sqrt(rr2);
    double w, dw;
    kern_wdw<double>(rr, P.inv_l, P.ad, w, dw);
    const double w2 = kern_w2(rr, P.inv_l, P.ad);
    const double f = -dw / rr, fp = (dw - w2 * rr) / rr2;
    double gw[D], gt[D], q[M], pv[M], rg = 0.0, rgg = 0.0;
    for (int K = 0; K < D; ++K) gw[K] = f * r[K];
    for (int K = 0; K < D; ++K) {
        double s2 = 0.0;
        for (int L2 = 0; L2 < D; ++L2) s2 += ld(SL::L + K * D + L2) * gw[L2];
        gt[K] = s2;
        rg += r[K] * s2;
        rgg += r[K] * ld(SL::G + K);
    }
    const double F = rg / (rr2 * rr2), e = dphi - rgg;
    qvec_d<D>(r, q);
    double qbd = 0.0, xp = 0.0;
    for (int a = 0; a < M; ++a) {
        double s2 = 0.0;
        for (int K = 0; K < D; ++K) s2 += ld(SL::C + K * M + a) * r[K];
        pv[a] = q[a] - s2;
        qbd += q[a] * ld(SL::BB + a);
    }
    for (int a = 0; a < M; ++a) xp += ld(SL::X + a) * pv[a];
    const double Fb = V * qbd * (e - xp), eb = V * F * qbd;
    double qb[M], pb[M];
    for (int a = 0; a < M; ++a) {
        pb[a] = -V * F * qbd * ld(SL::X + a);
        qb[a] = V * F * (e - xp) * ld(SL::BB + a) + pb[a];
    }
    for (int K = 0; K < D; ++K) {   // from e, p, F (rho and r.gt)
        double s2 = 0.0;
        for (int a = 0; a < M; ++a) s2 += ld(SL::C + K * M + a) * pb[a];
        rb[K] = -eb * ld(SL::G + K) - s2 + (-4.0 * rg / (rr2 * rr2 * rr) * Fb) * r[K] / rr +
                Fb / (rr2 * rr2) * gt[K];
    }
    // grad w's adjoint: L^T (rgbar r) + V dphi L^T gbar + V (L^T Cbar) q + V Bbar r
    const double rgb = Fb / (rr2 * rr2);
    double gwb[D];
    for (int K = 0; K < D; ++K) {
        double s2 = 0.0;
        for (int L2 = 0; L2 < D; ++L2)
            s2 += ld(SL::L + L2 * D + K) * rgb * r[L2] + V * ld(SL::BBAR + K * D + L2) * r[L2];
        s2 += V * dphi * ld(SL::GR + K);
        for (int a = 0; a < M; ++a) s2 += V * ld(SL::GQ + K * M + a) * q[a];
        gwb[K] = s2;
    }
    double rgw = 0.0;
    for (int K = 0; K < D; ++K) rgw += r[K] * gwb[K];
    for (int K = 0; K < D; ++K) rb[K] += f * gwb[K] + fp / rr * r[K] * rgw;   // H gwbar
    for (int a = 0; a < M; ++a) {   // q's adjoint, with V (L^T Cbar)^T grad w
        double s2 = 0.0;
        for (int K = 0; K < D; ++K) s2 += ld(SL::GQ + K * M + a) * gw[K];
        qb[a] += V * s2;
    }
    double qj[D];
    qjac_t<D>(r, qb, qj);
    for (int K = 0; K < D; ++K) {
        double s2 = 0.0;
        for (int L2 = 0; L2 < D; ++L2) s2 += ld(SL::BBAR + L2 * D + K) * gw[L2];
        rb[K] += qj[K] + V * s2;
    }
}

template <int D, bool PPE>
__global__ void __launch_bounds__(128) k_d2pos_b(DevParams P, const Part c, Work W, int n,
                                                 const double *phi, const double *scr,
                                                 double *xh_bar)
{
    if (step_failed(W.status)) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t cap = W.cap;
    const int tk = c.type[k], ok = c.orig[k];
    double out[D];
    for (int K = 0; K < D; ++K) out[K] = 0.0;
    if (tk != VIRTUAL) {
        double xk[3];
        load_hat<D>(c, k, xk);
        const int cnt = W.nbr_cnt[k];
        for (int q = 0; q < cnt; ++q) {
            const int m = W.nbr[(int64_t)q * cap + k];
            const int tm = c.type[m];
            if (tm == VIRTUAL || (tk != FLUID && tm != FLUID)) continue;
            double xm[3], r[D], rn[D], rr2 = 0.0;
            load_hat<D>(c, m, xm);
            for (int K = 0; K < D; ++K) {
                r[K] = xm[K] - xk[K];
                rn[K] = -r[K];
                rr2 += r[K] * r[K];
            }
            if (rr2 == 0.0) continue;
            double rb[D];
            if (tk == FLUID) {   // pair (k, m)
                d2pos_pair<D>(P, scr, cap, k, d2pos_dphi<D>(c, W, PPE, phi, k, m), r, W.vol[m], rb);
                for (int K = 0; K < D; ++K) out[K] -= rb[K];
            }
            if (tm == FLUID) {   // pair (m, k)
                d2pos_pair<D>(P, scr, cap, m, d2pos_dphi<D>(c, W, PPE, phi, m, k), rn, W.vol[k], rb);
                for (int K = 0; K < D; ++K) out[K] += rb[K];
            }
        }
    }
    for (int K = 0; K < D; ++K) xh_bar[(int64_t)K * n + ok] = out[K];
}

void launch_d2pos(const DevParams &P, Part cur, Work W, int64_t n, bool ppe, const double *phi,
                  const double *wbar, double *xh_bar, cudaStream_t st)
{
    // scratch: the pressure-equation coefficients' storage (>= 32 doubles per
    // particle in 2-D, 80 in 3-D in either form; the next step rebuilds it)
    double *scr = P.precision == VCT_MIXED ? (double *)W.pvalf : W.pval;
    const unsigned g = (unsigned)((n + 127) / 128);
    if (P.dim == 2) {
        if (ppe) {
            k_d2pos_a<2, true><<<g, 128, 0, st>>>(P, cur, W, (int)n, phi, wbar, scr);
            k_d2pos_b<2, true><<<g, 128, 0, st>>>(P, cur, W, (int)n, phi, scr, xh_bar);
        } else {
            k_d2pos_a<2, false><<<g, 128, 0, st>>>(P, cur, W, (int)n, phi, wbar, scr);
            k_d2pos_b<2, false><<<g, 128, 0, st>>>(P, cur, W, (int)n, phi, scr, xh_bar);
        }
    } else {
        if (ppe) {
            k_d2pos_a<3, true><<<g, 128, 0, st>>>(P, cur, W, (int)n, phi, wbar, scr);
            k_d2pos_b<3, true><<<g, 128, 0, st>>>(P, cur, W, (int)n, phi, scr, xh_bar);
        } else {
            k_d2pos_a<3, false><<<g, 128, 0, st>>>(P, cur, W, (int)n, phi, wbar, scr);
            k_d2pos_b<3, false><<<g, 128, 0, st>>>(P, cur, W, (int)n, phi, scr, xh_bar);
        }
    }
}


// ---------------------------------------------------------------------------
// a12 (part): derivative of the density estimate rho^_i = rho (sum_j V0 w_ij +
// V0 w(0)) (Sec. 4.4.2's <rho^>, over every neighbour type) with respect to the
// projected positions, neighbour sets fixed: d rho^_i / d r_j = rho V0 w'(rho_ij)
// r_ij / rho_ij for j != i (r_ij = r_j - r_i) and minus their sum for r_i.  For
// the loss sum_i rhobar_i rho^_i (fluid i) particle k gathers, over its
// neighbours m, rho V0 w' r_mk / rho_mk (rhobar_m [m fluid] + rhobar_k [k
// fluid]).  FP64.
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(128) k_rhopos(DevParams P, const Part c, Work W, int n,
                                                const double *rho_bar, double *xh_bar)
{
    if (step_failed(W.status)) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t cap = W.cap;
    const int ok = c.orig[k];
    const double bk = c.type[k] == FLUID ? rho_bar[ok] : 0.0;
    double xk[3], out[D];
    load_hat<D>(c, k, xk);
    for (int K = 0; K < D; ++K) out[K] = 0.0;
    const int cnt = W.nbr_cnt[k];
    for (int q = 0; q < cnt; ++q) {
        const int m = W.nbr[(int64_t)q * cap + k];
        const double bm = c.type[m] == FLUID ? rho_bar[c.orig[m]] : 0.0;
        if (bk == 0.0 && bm == 0.0) continue;
        double xm[3], r[D], rr2 = 0.0;
        load_hat<D>(c, m, xm);
        for (int K = 0; K < D; ++K) {
            r[K] = xk[K] - xm[K];   // r_mk
            rr2 += r[K] * r[K];
        }
        if (rr2 == 0.0) continue;
        const double rr = sqrt(rr2);
        double w, dw;
        kern_wdw<double>(rr, P.inv_l, P.ad, w, dw);
        const double s = P.rho * P.V0 * dw / rr * (bm + bk);
        for (int K = 0; K < D; ++K) out[K] += s * r[K];
    }
    for (int K = 0; K < D; ++K) xh_bar[(int64_t)K * n + ok] = out[K];
}

void launch_rhopos(const DevParams &P, Part cur, Work W, int64_t n, const double *rho_bar,
                   double *xh_bar, cudaStream_t st)
{
    const unsigned g = (unsigned)((n + 127) / 128);
    if (P.dim == 2) k_rhopos<2><<<g, 128, 0, st>>>(P, cur, W, (int)n, rho_bar, xh_bar);
    else k_rhopos<3><<<g, 128, 0, st>>>(P, cur, W, (int)n, rho_bar, xh_bar);
}

// ---------------------------------------------------------------------------
// a11: the stages of an ensemble step, each as one launch over all scenarios.
// Block b of a launch belongs to the scenario k with bs[k] <= b < bs[k + 1];
// it copies the part of that scenario's StageJob its stage reads into shared
// memory and runs the stage's body as block b - bs[k] of the scenario's own
// launch: every scenario runs the same device code as its own launch of the
// stage (the two kernels are compiled separately, so the compiler may fuse a
// multiply and an add differently: results agree to rounding).
// ---------------------------------------------------------------------------
// Blocks of 128 per SM the light batched stages (smoothing, wall velocities,
// right side, corrector, regularisation) are compiled for: their parameters come
// from shared memory instead of the kernel-parameter bank, which costs registers
// (64 ensemble scenarios, per step: right side 0.797 -> 0.726 ms, corrector
// 0.763 -> 0.698, regularisation 2.287 -> 2.230 at 8 blocks against 1)
#ifndef VCT_BATCH_LIGHT_MINB
#define VCT_BATCH_LIGHT_MINB 8
#endif
constexpr int BATCH_LIGHT_MINB = VCT_BATCH_LIGHT_MINB;
// ... and the 2-D passes (pass 2 at 4 blocks: 3.67 -> 3.30 ms per ensemble step;
// pass 1 at 2 blocks: no change)
#ifndef VCT_BATCH_PASS1_MINB2
#define VCT_BATCH_PASS1_MINB2 1
#endif
#ifndef VCT_BATCH_PASS2_MINB2
#define VCT_BATCH_PASS2_MINB2 4
#endif
constexpr int BATCH_PASS1_MINB2 = VCT_BATCH_PASS1_MINB2, BATCH_PASS2_MINB2 = VCT_BATCH_PASS2_MINB2;
static_assert(offsetof(StageJob, P) % 16 == 0 && offsetof(StageJob, alt) % 16 == 0 &&
                  offsetof(StageJob, M) % 16 == 0 && sizeof(StageJob) % 16 == 0,
              "StageJob prefixes are copied in 16-byte words");
constexpr int SJ_CW = (int)offsetof(StageJob, P);      // n, cur, W
constexpr int SJ_CWP = (int)offsetof(StageJob, alt);   // + P
constexpr int SJ_CWPA = (int)offsetof(StageJob, M);    // + alt
constexpr int SJ_ALL = (int)sizeof(StageJob);          // + M

template <class F>
__global__ void __launch_bounds__(F::NT, F::MINB) k_batched(const StageJob *__restrict__ jobs,
                                                            const int *__restrict__ bs, int njobs, F f)
{
    __shared__ int4 sj[F::BYTES / 16];
    const int b = (int)blockIdx.x;
    int lo = 0, hi = njobs;   // bs[lo] <= b < bs[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(bs + mid) <= b) lo = mid;
        else hi = mid;
    }
    const int4 *src = reinterpret_cast<const int4 *>(jobs + lo);
    for (int k = threadIdx.x; k < F::BYTES / 16; k += blockDim.x) sj[k] = __ldg(src + k);
    __syncthreads();
    f(*reinterpret_cast<const StageJob *>(sj), b - __ldg(bs + lo));
}

struct BZero {   // the counters a step starts from: cell counts and cursors, row counts, barrier
    static constexpr int NT = 256, MINB = 1, BYTES = SJ_CW;
    __device__ void operator()(const StageJob &j, int b) const
    {
        const int64_t i = (int64_t)b * NT + threadIdx.x;
        if (i <= j.W.ncell) j.W.cell_count[i] = 0;
        if (i < j.W.ncell) j.W.cursor[i] = 0;
        if (i < 2) {
            j.W.counts[i] = 0;
            j.W.bar[i] = 0u;
        }
    }
};
struct BMapKey {
    static constexpr int NT = 256, MINB = 1, BYTES = SJ_CWP;
    __device__ void operator()(const StageJob &j, int b) const { map_key_body(j.P, j.cur, j.W, (int)j.n, b); }
};
// exclusive scans: of the cell counts (CELLS) or of the unknown-row flags
template <bool CELLS>
__device__ __forceinline__ void scan_args(const StageJob &j, const int32_t *&in, int32_t *&out, int64_t &m)
{
    in = CELLS ? j.W.cell_count : j.W.urow_flag;
    out = CELLS ? j.W.cell_start : j.W.urow_pos;
    m = CELLS ? j.W.ncell : j.n;
}
template <bool CELLS>
struct BScanBlocks {
    static constexpr int NT = SCAN_T, MINB = 1, BYTES = SJ_CW;
    __device__ void operator()(const StageJob &j, int b) const
    {
        const int32_t *in;
        int32_t *out;
        int64_t m;
        scan_args<CELLS>(j, in, out, m);
        scan_blocks_body<int32_t>(in, out, j.W.scan_tmp, m, b);
    }
};
template <bool CELLS>
struct BScanTops {
    static constexpr int NT = SCAN_T, MINB = 1, BYTES = SJ_CW;
    __device__ void operator()(const StageJob &j, int b) const
    {
        const int32_t *in;
        int32_t *out;
        int64_t m;
        scan_args<CELLS>(j, in, out, m);
        int64_t nb = (m + SCAN_B - 1) / SCAN_B;
        if (nb == 0) nb = 1;
        scan_tops_body<int32_t>(j.W.scan_tmp, nb, out, m, b);
    }
};
template <bool CELLS>
struct BScanAdd {
    static constexpr int NT = 256, MINB = 1, BYTES = SJ_CW;
    __device__ void operator()(const StageJob &j, int b) const
    {
        const int32_t *in;
        int32_t *out;
        int64_t m;
        scan_args<CELLS>(j, in, out, m);
        scan_add_body<int32_t>(out, j.W.scan_tmp, m, b);
    }
};
struct BScatter {
    static constexpr int NT = 256, MINB = 1, BYTES = SJ_CW;
    __device__ void operator()(const StageJob &j, int b) const { scatter_body(j.W, j.cur, (int)j.n, b); }
};
struct BCellSort {
    static constexpr int NT = 128, MINB = 1, BYTES = SJ_CW;
    __device__ void operator()(const StageJob &j, int b) const { cell_sort_body(j.W, j.cur, j.W.ncell, b); }
};
struct BReorder {
    static constexpr int NT = 256, MINB = 1, BYTES = SJ_CWPA;
    __device__ void operator()(const StageJob &j, int b) const { reorder_body(j.cur, j.alt, j.W, (int)j.n, j.P, b); }
};
template <int D, typename R>
struct BNeighbours {
    static constexpr int NT = 128, MINB = 1, BYTES = SJ_CWP;
    __device__ void operator()(const StageJob &j, int b) const { neighbours_body<D>(j.P, j.cur, j.W, (int)j.n, b); }
};
template <int D, typename R>
struct BSmoothing {
    static constexpr int NT = 128, MINB = BATCH_LIGHT_MINB, BYTES = SJ_CWP;
    __device__ void operator()(const StageJob &j, int b) const { smoothing_body<D, R>(j.P, j.cur, j.W, (int)j.n, b); }
};
struct BJbarCopy {   // the smoothed Jbar into the state
    static constexpr int NT = 256, MINB = 1, BYTES = SJ_CW;
    __device__ void operator()(const StageJob &j, int b) const
    {
        const int64_t i = (int64_t)b * NT + threadIdx.x;
        if (i < j.n) j.cur.jbar[i] = j.W.jbar_tmp[i];
    }
};
template <int D, typename R>
struct BWallVelocity {
    static constexpr int NT = 128, MINB = BATCH_LIGHT_MINB, BYTES = SJ_CWP;
    __device__ void operator()(const StageJob &j, int b) const { wall_velocity_body<D>(j.P, j.cur, j.W, (int)j.n, b); }
};
template <int D, typename R>
struct BPass1 {
    static constexpr int NT = 128, MINB = D == 2 ? BATCH_PASS1_MINB2 : pass1_min_blocks<D>(), BYTES = SJ_CWP;
    __device__ void operator()(const StageJob &j, int b) const { pass1_body<D, R>(j.P, j.cur, j.W, (int)j.n, b); }
};
template <int D, typename R>
struct BPass2 {
    static constexpr int NT = 128, MINB = D == 2 ? BATCH_PASS2_MINB2 : pass2_min_blocks<D>(), BYTES = SJ_CWP;
    __device__ void operator()(const StageJob &j, int b) const { pass2_body<D, R>(j.P, j.cur, j.W, (int)j.n, 1, b); }
};
template <int D, typename R>
struct BPass2Isph {
    static constexpr int NT = 128, MINB = 1, BYTES = SJ_CWP;
    __device__ void operator()(const StageJob &j, int b) const { pass2_isph_body<D, R>(j.P, j.cur, j.W, (int)j.n, b); }
};
template <int D, typename R>
struct BRhs {
    static constexpr int NT = 128, MINB = BATCH_LIGHT_MINB, BYTES = SJ_CWP;
    __device__ void operator()(const StageJob &j, int b) const { rhs_body<D, R>(j.P, j.cur, j.W, (int)j.n, b); }
};
struct BUrowFlags {
    static constexpr int NT = 256, MINB = 1, BYTES = SJ_CW;
    __device__ void operator()(const StageJob &j, int b) const { urow_flags_body(j.W, (int)j.n, b); }
};
struct BUrowScatter {
    static constexpr int NT = 256, MINB = 1, BYTES = SJ_CW;
    __device__ void operator()(const StageJob &j, int b) const { urow_scatter_body(j.W, (int)j.n, b); }
};
struct BMgDsc {
    static constexpr int NT = 256, MINB = 1, BYTES = SJ_CW;
    __device__ void operator()(const StageJob &j, int b) const { mg_dsc_body(j.W, (int)j.n, b); }
};
template <int D, typename R>
struct BMgRowcell {
    static constexpr int NT = 256, MINB = 1, BYTES = SJ_ALL;
    __device__ void operator()(const StageJob &j, int b) const
    {
        mg_rowcell_body<D>(j.W, j.M, (int)j.n, j.P.precision == VCT_MIXED, b);
    }
};
template <int D, typename R>
struct BMgLevel1 {
    static constexpr int NT = 256, MINB = 1, BYTES = SJ_ALL;
    __device__ void operator()(const StageJob &j, int b) const
    {
        if (j.M.rowcell && !j.M.fly) mg_level1_rc_body<D>(j.W, j.M, b);
        else mg_level1_body<D>(j.W, j.M, j.P.precision == VCT_MIXED, b);
    }
};
template <int D, typename R>
struct BMgCoarsen {
    static constexpr int NT = 128, MINB = 1, BYTES = SJ_ALL;
    int l;
    __device__ void operator()(const StageJob &j, int b) const { mg_coarsen_body<D>(j.W, j.M, l, b); }
};
template <int D, typename R>
struct BMgCoarsenSmall {
    static constexpr int NT = 256, MINB = 1, BYTES = SJ_ALL;
    int small;   // the host's small-level size
    __device__ void operator()(const StageJob &j, int b) const
    {
        int l = 1;   // the first level the per-level launches did not build
        while (l < j.M.L && j.M.n[l + 1] > small) ++l;
        mg_coarsen_small_body<D>(j.W, j.M, l, b);
    }
};
template <int D, typename R, bool SUM>
struct BCorrector {
    static constexpr int NT = 128, MINB = BATCH_LIGHT_MINB, BYTES = SJ_CWP;
    __device__ void operator()(const StageJob &j, int b) const { corrector_body<D, R, SUM>(j.P, j.cur, j.W, (int)j.n, b); }
};
template <int D, typename R>
struct BCorrectorPlain : BCorrector<D, R, false> {};
template <int D, typename R>
struct BCorrectorSum : BCorrector<D, R, true> {};
template <int D, typename R>
struct BRegGeom {
    static constexpr int NT = 128, MINB = BATCH_LIGHT_MINB, BYTES = SJ_CWP;
    __device__ void operator()(const StageJob &j, int b) const { reg_geom_body<D>(j.P, j.cur, j.W, (int)j.n, b); }
};
template <int D, typename R>
struct BRegDs {
    static constexpr int NT = 128, MINB = BATCH_LIGHT_MINB, BYTES = SJ_CWP;
    __device__ void operator()(const StageJob &j, int b) const { reg_ds_body<D, R>(j.P, j.cur, j.W, (int)j.n, b); }
};
template <int D, typename R>
struct BRegApply {
    static constexpr int NT = 128, MINB = BATCH_LIGHT_MINB, BYTES = SJ_CWP;
    __device__ void operator()(const StageJob &j, int b) const { reg_apply_body<D, R>(j.P, j.cur, j.W, (int)j.n, b); }
};

int batch_coarsen_levels(const MG &M)
{
    int l = 1;
    while (l < M.L && M.n[l + 1] > small_level()) ++l;
    return l;   // BS_MG_COARSEN runs at levels 1 .. l - 1
}

int batch_stage_blocks(int s, const DevParams &P, const Work &W, const MG &M, int64_t n,
                       bool rows_list, int level)
{
    const int64_t nc = W.ncell;
    const int b256 = (int)((n + 255) / 256), b128 = (int)((n + 127) / 128);
    const bool smooth = P.kind == VCT_MAP_SIGMA && P.volume_mode == 2;
    const bool reg = regularise_on(P);
    const int lend = batch_coarsen_levels(M);
    int64_t snb;
    switch (s) {
    case BS_ZERO: return (int)((nc + 1 + 255) / 256);
    case BS_MAP_KEY: case BS_SCATTER: case BS_REORDER: case BS_MG_DSC: return b256;
    case BS_CSCAN_BLOCKS:
        snb = (nc + SCAN_B - 1) / SCAN_B;
        return snb == 0 ? 1 : (int)snb;
    case BS_CSCAN_TOPS: return 1;
    case BS_CSCAN_ADD: return (int)((nc + 255) / 256);
    case BS_CELL_SORT: return (int)((nc + 127) / 128);
    case BS_NEIGHBOURS: case BS_PASS1: case BS_RHS: return b128;
    case BS_SMOOTHING: return smooth ? b128 : 0;
    case BS_JBAR_COPY: return smooth ? b256 : 0;
    case BS_WALL_VELOCITY: return P.slip ? b128 : 0;
    case BS_PASS2: return P.operators == 1 ? 0 : b128;
    case BS_PASS2_ISPH: return P.operators == 1 ? b128 : 0;
    case BS_UROW_FLAGS: case BS_RSCAN_ADD: case BS_UROW_SCATTER: return rows_list ? b256 : 0;
    case BS_RSCAN_BLOCKS:
        snb = (n + SCAN_B - 1) / SCAN_B;
        return rows_list ? (snb == 0 ? 1 : (int)snb) : 0;
    case BS_RSCAN_TOPS: return rows_list ? 1 : 0;
    case BS_MG_ROWCELL: return mg_rowcell_on(M) ? (int)((n * (P.dim == 2 ? 4 : 8) + 255) / 256) : 0;
    case BS_MG_LEVEL1:
        return mg_rowcell_on(M) ? (int)(((int64_t)M.n[1] + 255) / 256)
                                : (int)(((int64_t)M.n[1] * 32 + 255) / 256);
    case BS_MG_COARSEN: return level >= 1 && level < lend ? (M.n[level + 1] + 127) / 128 : 0;
    case BS_MG_COARSEN_SMALL: return lend < M.L ? 1 : 0;
    case BS_CORRECTOR: return P.operators == 1 ? 0 : b128;
    case BS_CORRECTOR_SUM: return P.operators == 1 ? b128 : 0;
    case BS_REG_GEOM: case BS_REG_APPLY: return reg ? b128 : 0;
    case BS_REG_DS: return reg && P.ds_overlap > 0.0 ? b128 : 0;
    default: return 0;
    }
}

template <class F>
static void run_batched(const StageJob *jobs, const int *bs, int njobs, int total, F f, cudaStream_t st)
{
    k_batched<F><<<(unsigned)total, F::NT, 0, st>>>(jobs, bs, njobs, f);
}

// the functor template FT<D, R> of the batch's dimension and precision
template <template <int, typename> class FT, class... A>
static void run_dr(int dim, bool mixed, const StageJob *jobs, const int *bs, int njobs, int total,
                   cudaStream_t st, A... a)
{
    if (dim == 2) {
        if (mixed) run_batched(jobs, bs, njobs, total, FT<2, float>{a...}, st);
        else run_batched(jobs, bs, njobs, total, FT<2, double>{a...}, st);
    } else {
        if (mixed) run_batched(jobs, bs, njobs, total, FT<3, float>{a...}, st);
        else run_batched(jobs, bs, njobs, total, FT<3, double>{a...}, st);
    }
}

void launch_batched(int s, int dim, int precision, const StageJob *jobs, const int *bs, int njobs,
                    int total, int level, cudaStream_t st)
{
    if (total <= 0) return;
    const bool mx = precision == VCT_MIXED;
    switch (s) {
    case BS_ZERO: run_batched(jobs, bs, njobs, total, BZero{}, st); break;
    case BS_MAP_KEY: run_batched(jobs, bs, njobs, total, BMapKey{}, st); break;
    case BS_CSCAN_BLOCKS: run_batched(jobs, bs, njobs, total, BScanBlocks<true>{}, st); break;
    case BS_CSCAN_TOPS: run_batched(jobs, bs, njobs, total, BScanTops<true>{}, st); break;
    case BS_CSCAN_ADD: run_batched(jobs, bs, njobs, total, BScanAdd<true>{}, st); break;
    case BS_SCATTER: run_batched(jobs, bs, njobs, total, BScatter{}, st); break;
    case BS_CELL_SORT: run_batched(jobs, bs, njobs, total, BCellSort{}, st); break;
    case BS_REORDER: run_batched(jobs, bs, njobs, total, BReorder{}, st); break;
    case BS_NEIGHBOURS: run_dr<BNeighbours>(dim, mx, jobs, bs, njobs, total, st); break;
    case BS_SMOOTHING: run_dr<BSmoothing>(dim, mx, jobs, bs, njobs, total, st); break;
    case BS_JBAR_COPY: run_batched(jobs, bs, njobs, total, BJbarCopy{}, st); break;
    case BS_WALL_VELOCITY: run_dr<BWallVelocity>(dim, mx, jobs, bs, njobs, total, st); break;
    case BS_PASS1: run_dr<BPass1>(dim, mx, jobs, bs, njobs, total, st); break;
    case BS_PASS2: run_dr<BPass2>(dim, mx, jobs, bs, njobs, total, st); break;
    case BS_PASS2_ISPH: run_dr<BPass2Isph>(dim, mx, jobs, bs, njobs, total, st); break;
    case BS_RHS: run_dr<BRhs>(dim, mx, jobs, bs, njobs, total, st); break;
    case BS_UROW_FLAGS: run_batched(jobs, bs, njobs, total, BUrowFlags{}, st); break;
    case BS_RSCAN_BLOCKS: run_batched(jobs, bs, njobs, total, BScanBlocks<false>{}, st); break;
    case BS_RSCAN_TOPS: run_batched(jobs, bs, njobs, total, BScanTops<false>{}, st); break;
    case BS_RSCAN_ADD: run_batched(jobs, bs, njobs, total, BScanAdd<false>{}, st); break;
    case BS_UROW_SCATTER: run_batched(jobs, bs, njobs, total, BUrowScatter{}, st); break;
    case BS_MG_DSC: run_batched(jobs, bs, njobs, total, BMgDsc{}, st); break;
    case BS_MG_ROWCELL: run_dr<BMgRowcell>(dim, mx, jobs, bs, njobs, total, st); break;
    case BS_MG_LEVEL1: run_dr<BMgLevel1>(dim, mx, jobs, bs, njobs, total, st); break;
    case BS_MG_COARSEN: run_dr<BMgCoarsen>(dim, mx, jobs, bs, njobs, total, st, level); break;
    case BS_MG_COARSEN_SMALL: run_dr<BMgCoarsenSmall>(dim, mx, jobs, bs, njobs, total, st, small_level()); break;
    case BS_CORRECTOR: run_dr<BCorrectorPlain>(dim, mx, jobs, bs, njobs, total, st); break;
    case BS_CORRECTOR_SUM: run_dr<BCorrectorSum>(dim, mx, jobs, bs, njobs, total, st); break;
    case BS_REG_GEOM: run_dr<BRegGeom>(dim, mx, jobs, bs, njobs, total, st); break;
    case BS_REG_DS: run_dr<BRegDs>(dim, mx, jobs, bs, njobs, total, st); break;
    case BS_REG_APPLY: run_dr<BRegApply>(dim, mx, jobs, bs, njobs, total, st); break;
    default: break;
    }
}

}  // namespace vct

// ===========================================================================
// Allocation-free neighbour search: vct_build_neighbours_noalloc.
//
// Some callers cannot allocate device memory at the moment they need neighbour
// lists: an application that has handed all device memory to its own pool
// allocator (a further cudaMalloc fails or breaks its accounting), or a loop
// with a latency budget that cannot afford cudaMalloc/cudaFree, which may
// synchronise the device.  Such callers also cannot own a vct_ctx, whose
// vct_init allocates.  For them this entry point takes the map and parameters
// directly and keeps all of its scratch in the file-scope array below, sized
// for at most NA_MAX_PARTICLES particles and NA_MAX_CELLS cells (about 1 MB).
// Every GPU that loads this library holds that array until the process exits.
//
// The array is shared by every call on a device and keeps the last call's
// contents; each call clears the counters it needs before use.  Calls that
// overlap on the GPU (for example on two streams at once) race on the array
// and must not be issued.
// ===========================================================================
namespace vct_noalloc {

constexpr int NA_MAX_PARTICLES = 16384;
constexpr int NA_MAX_CELLS = 32768;

struct Scratch {
    double xh[3][NA_MAX_PARTICLES];     // projected positions, caller order
    int32_t key[NA_MAX_PARTICLES];      // cell of each particle
    int32_t perm[NA_MAX_PARTICLES];     // particles ordered by cell, then by index
    int32_t row_cnt[NA_MAX_PARTICLES];  // neighbours of each particle
    int32_t cell_count[NA_MAX_CELLS + 1];
    int32_t cell_start[NA_MAX_CELLS + 1];
    int32_t cursor[NA_MAX_CELLS];
    int32_t status[4];                  // [0]: 0 or VCT_ERR_CAPACITY
};

}  // namespace vct_noalloc

static __device__ __align__(256) vct_noalloc::Scratch g_noalloc_scratch;

namespace vct_noalloc {

using vct::DevParams;

__global__ void k_na_clear(Scratch *S, int ncell)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= ncell; c += gridDim.x * blockDim.x) {
        S->cell_count[c] = 0;
        if (c < ncell) S->cursor[c] = 0;
        if (c < 4) S->status[c] = 0;
    }
}

__global__ void k_na_map(DevParams P, vct_state s, int n, Scratch *S)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double y = P.dim == 3 ? s.y[i] : 0.0, zh, J, sx, sy, c0, c3;
    vct::map_metric(P, s.x[i], y, s.z[i], zh, J, sx, sy, c0, c3);
    S->xh[0][i] = s.x[i];
    S->xh[1][i] = y;
    S->xh[2][i] = zh;
    int cx = vct::cell_coord(P, s.x[i], 0);
    int cy = P.dim == 3 ? vct::cell_coord(P, y, 1) : 0;
    int cz = vct::cell_coord(P, zh, 2);
    int key = (cz * P.nc[1] + cy) * P.nc[0] + cx;
    S->key[i] = key;
    atomicAdd(&S->cell_count[key], 1);
}

// Exclusive scan by one block of 1024 threads; out[m] = total.
template <typename TO>
__device__ void na_block_scan(const int32_t *in, TO *out, int m)
{
    __shared__ long long sh[1024];
    const int t = threadIdx.x, per = (m + 1023) / 1024;
    const int a = t * per, b = min(a + per, m);
    long long loc = 0;
    for (int k = a; k < b; ++k) loc += in[k];
    sh[t] = loc;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        long long v = t >= o ? sh[t - o] : 0;
        __syncthreads();
        sh[t] += v;
        __syncthreads();
    }
    long long run = sh[t] - loc;
    for (int k = a; k < b; ++k) {
        out[k] = (TO)run;
        run += in[k];
    }
    if (t == 1023) out[m] = (TO)sh[1023];
}

__global__ void k_na_scan_cells(Scratch *S, int ncell)
{
    na_block_scan<int32_t>(S->cell_count, S->cell_start, ncell);
}

__global__ void k_na_scatter(Scratch *S, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int key = S->key[i];
    S->perm[S->cell_start[key] + atomicAdd(&S->cursor[key], 1)] = i;
}

__global__ void k_na_cell_sort(Scratch *S, int ncell)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    int a = S->cell_start[c], b = S->cell_start[c + 1];
    for (int k = a + 1; k < b; ++k) {
        int v = S->perm[k], m = k - 1;
        while (m >= a && S->perm[m] > v) {
            S->perm[m + 1] = S->perm[m];
            --m;
        }
        S->perm[m + 1] = v;
    }
}

// Visit the candidates of particle i (3^d cells) and apply the FP64 predicate
// without FMA; fn(j) is called for every neighbour.
template <typename Fn>
__device__ void na_visit(const DevParams &P, const Scratch *S, int i, Fn fn)
{
    const double xi = S->xh[0][i], yi = S->xh[1][i], zi = S->xh[2][i];
    int cx = vct::cell_coord(P, xi, 0);
    int cy = P.dim == 3 ? vct::cell_coord(P, yi, 1) : 0;
    int cz = vct::cell_coord(P, zi, 2);
    const int ylo = P.dim == 3 ? -1 : 0, yhi = P.dim == 3 ? 1 : 0;
    for (int dz = -1; dz <= 1; ++dz) {
        int z2 = cz + dz;
        if (z2 < 0 || z2 >= P.nc[2]) continue;
        for (int dy = ylo; dy <= yhi; ++dy) {
            int y2 = cy + dy;
            if (y2 < 0 || y2 >= P.nc[1]) continue;
            int row = (z2 * P.nc[1] + y2) * P.nc[0];
            int xa = cx > 0 ? cx - 1 : 0, xb = cx + 1 < P.nc[0] ? cx + 1 : P.nc[0] - 1;
            for (int k = S->cell_start[row + xa]; k < S->cell_start[row + xb + 1]; ++k) {
                int j = S->perm[k];
                if (j == i) continue;
                double dx = __dsub_rn(S->xh[0][j], xi), dz2 = __dsub_rn(S->xh[2][j], zi), d2;
                if (P.dim == 2) {
                    d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dz2, dz2));
                } else {
                    double dy2 = __dsub_rn(S->xh[1][j], yi);
                    d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy2, dy2)),
                                   __dmul_rn(dz2, dz2));
                }
                if (d2 < P.re2) fn(j);
            }
        }
    }
}

__global__ void k_na_count(DevParams P, Scratch *S, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int cnt = 0;
    na_visit(P, S, i, [&](int) { ++cnt; });
    S->row_cnt[i] = cnt;
}

__global__ void k_na_scan_rows(Scratch *S, int n, int64_t *row_ptr)
{
    na_block_scan<int64_t>(S->row_cnt, row_ptr, n);
}

__global__ void k_na_fill(DevParams P, Scratch *S, int n, const int64_t *row_ptr, int32_t *col,
                          int64_t col_cap)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (row_ptr[n] > col_cap) {
        if (i == 0) S->status[0] = VCT_ERR_CAPACITY;
        return;
    }
    int32_t *out = col + row_ptr[i];
    int cnt = 0;
    na_visit(P, S, i, [&](int j) {   // insertion into the row, ascending index
        int m = cnt - 1;
        while (m >= 0 && out[m] > j) {
            out[m + 1] = out[m];
            --m;
        }
        out[m + 1] = j;
        ++cnt;
    });
}

// Address of the scratch array on the current device, set up once per device.
vct_status scratch_on_device(Scratch **out)
{
    static Scratch *ptr[128] = {};
    static std::mutex mu;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return VCT_ERR_CUDA;
    std::lock_guard<std::mutex> lock(mu);
    if (!ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) return VCT_ERR_CUDA;
        ptr[dev] = (Scratch *)p;
    }
    *out = ptr[dev];
    return VCT_OK;
}

}  // namespace vct_noalloc

extern "C" __attribute__((visibility("default"))) vct_status vct_build_neighbours_noalloc(
    const vct_bathymetry *bathy, vct_map_kind kind, double aspect_ratio, const vct_params *prm,
    const vct_state *s, int64_t *row_ptr, int32_t *col, int64_t col_cap, int64_t *nnz,
    void *stream)
{
    using namespace vct_noalloc;
    if (!bathy || !prm || !s || !row_ptr || !nnz) return VCT_ERR_ARG;
    if (prm->dim != 2 && prm->dim != 3) return VCT_ERR_ARG;
    if ((int)kind < 0 || (int)kind > 3) return VCT_ERR_ARG;
    if (!(prm->d0 > 0) || bathy->n_gauss < 0 || bathy->n_gauss > VCT_MAX_GAUSS) return VCT_ERR_ARG;
    if (bathy->n_gauss > 0 && (!bathy->amp || !bathy->cx || !bathy->cy || !bathy->width))
        return VCT_ERR_ARG;
    if ((kind == VCT_MAP_E || kind == VCT_MAP_BFE) && !(aspect_ratio > 0)) return VCT_ERR_ARG;
    if (kind == VCT_MAP_SIGMA && !(prm->H_hat > 0 && prm->alpha_min > 0 &&
                                   prm->alpha_max >= prm->alpha_min))
        return VCT_ERR_ARG;
    if (!s->x || !s->z || (prm->dim == 3 && !s->y)) return VCT_ERR_ARG;
    if (s->n <= 0) return VCT_ERR_ARG;
    if (s->n > NA_MAX_PARTICLES) return VCT_ERR_CAPACITY;
    const int n = (int)s->n;
    vct::DevParams P;
    memset(&P, 0, sizeof P);
    P.dim = prm->dim;
    P.kind = (int)kind;
    P.n_gauss = bathy->n_gauss;
    P.aspect = aspect_ratio;
    P.d0 = prm->d0;
    P.l = prm->l_over_d0 * prm->d0;
    P.re = prm->re_over_l * P.l;
    P.re2 = P.re * P.re;
    P.H = prm->H;
    P.H_hat = prm->H_hat;
    P.amin = prm->alpha_min;
    P.amax = prm->alpha_max;
    P.cell_h = P.re;
    P.inv_cell_h = 1.0 / P.cell_h;
    int64_t ncell = 1;
    {
        vct_status gs = vct::cell_grid(prm, P.re, NA_MAX_CELLS, P.nc, &ncell);
        if (gs != VCT_OK) return gs;
    }
    for (int k = 0; k < 3; ++k) P.box_lo[k] = prm->box_lo[k];
    P.h0 = bathy->h0;
    P.slope_x = bathy->slope_x;
    P.slope_y = bathy->slope_y;
    P.cos_amp = bathy->cos_amp;
    P.cos_len = bathy->cos_len;
    for (int g = 0; g < bathy->n_gauss; ++g) {
        P.gamp[g] = bathy->amp[g];
        P.gcx[g] = bathy->cx[g];
        P.gcy[g] = bathy->cy[g];
        P.gwid[g] = bathy->width[g];
        P.ginv2[g] = 1.0 / (bathy->width[g] * bathy->width[g]);
    }
    Scratch *S = nullptr;
    vct_status v = scratch_on_device(&S);
    if (v) return v;
    cudaStream_t st = (cudaStream_t)stream;
    // An error the calling thread left pending (from earlier work, e.g. its
    // framework's) stays pending for its owner: this call neither clears it
    // nor reports it as its own.  Launch errors of this call are detected
    // when nothing was pending at entry.
    const bool clean_at_entry = cudaPeekAtLastError() == cudaSuccess;
    const int nc = (int)ncell, gp = (n + 255) / 256, gc = (nc + 255) / 256;
    k_na_clear<<<gc + 1, 256, 0, st>>>(S, nc);
    k_na_map<<<gp, 256, 0, st>>>(P, *s, n, S);
    k_na_scan_cells<<<1, 1024, 0, st>>>(S, nc);
    k_na_scatter<<<gp, 256, 0, st>>>(S, n);
    k_na_cell_sort<<<gc, 256, 0, st>>>(S, nc);
    k_na_count<<<gp, 256, 0, st>>>(P, S, n);
    k_na_scan_rows<<<1, 1024, 0, st>>>(S, n, row_ptr);
    if (col) k_na_fill<<<gp, 256, 0, st>>>(P, S, n, row_ptr, col, col_cap);
    if (clean_at_entry && cudaPeekAtLastError() != cudaSuccess) {
        (void)cudaGetLastError();   // this call's own launch error
        return VCT_ERR_CUDA;
    }
    int64_t total = 0;
    int32_t status = 0;
    cudaError_t e = cudaMemcpyAsync(&total, row_ptr + n, sizeof total, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&status, S->status, sizeof status, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return VCT_ERR_CUDA;
    *nnz = total;
    if (col && total > col_cap) return VCT_ERR_CAPACITY;
    return (vct_status)status;
}
