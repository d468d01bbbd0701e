// goc_aux.cuh -- metric precompute (FP64), initial state, moment export and
// FP64 reductions.
#pragma once

#include "goc_aa.cuh"
#include "goc_device.cuh"
#include "goc_step.cuh"

namespace goc {

// ---- metric factors of one axis in FP64 (Sec. 6; Eq. metricfactor,
// Eq. curvaturematrix).  Entries 0..n-1 are the nodes, n and n+1 the walls
// at xi = 0 and xi = n.
struct MapParams {
    int kind;          // 0 uniform, 1 tanh2, 2 sine, 3 roberts, 4 tanh1 (one wall), 5 sinh (interior), 6 annulus
    int n, periodic;
    double beta, a, gamma, alpha, mu, yc;
    double r_in, r_out, sectors;   // annulus (xi1 axis)
    int n2;                        // annulus: nodes along xi2
};

__device__ void map_h_theta(const MapParams &m, double xi, double &h, double &th) {
    const double n = (double)m.n;
    if (m.kind == 0 || (m.kind == 1 && m.beta == 0.0)) {
        h = 1.0;
        th = 0.0;
    } else if (m.kind == 1) {   // Eq. metriccoefficient with cell-centred nodes, L = n
        const double arg = m.beta * (2.0 * xi / n - 1.0);
        const double ch = cosh(arg);
        const double sech2 = 1.0 / (ch * ch);
        h = m.beta / tanh(m.beta) * sech2;
        th = -(4.0 * tanh(m.beta) / n) * tanh(arg) / sech2;
    } else if (m.kind == 2) {   // periodic sine stretching
        const double ph = 2.0 * 3.14159265358979323846 * xi / n;
        h = 1.0 + m.a * cos(ph);
        th = -m.a * (2.0 * 3.14159265358979323846 / n) * sin(ph) / (h * h);
    } else if (m.kind == 4) {   // one wall (Eq. metriccoefficientB), clustered at xi = 0
        const double arg = m.beta * (1.0 - xi / n);
        const double ch = cosh(arg);
        const double sech2 = 1.0 / (ch * ch);
        h = m.beta / tanh(m.beta) * sech2;
        th = (2.0 * tanh(m.beta) / n) * tanh(arg) / sech2;
    } else if (m.kind == 5) {   // interior point (Eq. B_Holst, Eq. h_2_Holst)
        const double B = log((1.0 + (exp(m.mu) - 1.0) * m.yc) / (1.0 + (exp(-m.mu) - 1.0) * m.yc)) / (2.0 * m.mu);
        const double arg = m.mu * (xi / n - B), smb = sinh(m.mu * B), ch = cosh(arg);
        h = m.yc * m.mu * ch / smb;
        th = smb / (m.yc * n) * tanh(arg) / ch;
    } else {                    // Roberts (Eq. h2_Roberts), lambda = (gamma+1)/(gamma-1)
        const double lam = (m.gamma + 1.0) / (m.gamma - 1.0);
        const double s = (xi / n - m.alpha) / (1.0 - m.alpha);
        const double ls = pow(lam, s);
        h = (2.0 * m.gamma / (2.0 * m.alpha + 1.0)) * log(lam) / (1.0 - m.alpha) * ls / ((1.0 + ls) * (1.0 + ls));
        th = (1.0 / n) * ((1.0 + 2.0 * m.alpha) / (2.0 * m.gamma)) * (1.0 / ls - ls);
    }
}

__global__ void metric_axis_kernel(MapParams m, double *h, double *th) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m.n + 2) return;
    double xi;
    if (k < m.n) xi = m.periodic ? (double)k : (double)k + 0.5;
    else xi = (k == m.n) ? 0.0 : (double)m.n;
    double hv, tv;
    map_h_theta(m, xi, hv, tv);
    h[k] = hv;
    th[k] = tv;
}

// Annular sector (Sec. 8.1, Eq. 2_annularsector / 5_annularsector): rows
// h1, theta11, h2, theta21 as functions of xi1, each [n + 2] (nodes, then the
// walls xi1 = 0 and n); r = r_in exp(ln(r_out/r_in) xi1/n).
__global__ void annulus_metric_kernel(MapParams m, double *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m.n + 2) return;
    const double xi = k < m.n ? (double)k + 0.5 : (k == m.n ? 0.0 : (double)m.n);
    const double lam = log(m.r_out / m.r_in), r = m.r_in * exp(lam * xi / m.n);
    const int w = m.n + 2;
    out[k] = r * lam / m.n;
    out[w + k] = 1.0 / r;
    out[2 * w + k] = 2.0 * 3.14159265358979323846 * r / (m.sectors * m.n2);
    out[3 * w + k] = 1.0 / r;
}

// q = min over the nodes of both axes (Eq. GOC-LBE_CFL): one block.
__global__ void min_h_kernel(const double *h1, int n1, const double *h2, int n2, double *q) {
    __shared__ double red[32];
    double v = 1e300;
    for (int k = threadIdx.x; k < n1; k += blockDim.x) v = fmin(v, h1[k]);
    for (int k = threadIdx.x; k < n2; k += blockDim.x) v = fmin(v, h2[k]);
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 1e300;
        for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) *q = v;
    }
}

// FP32 tables of one axis from the FP64 metric: h, 1/h, theta, the pull
// corrections of the storage reference (see goc_step.cuh)
//   rm[k] = rho0 cs2 [ (1/h(k-1) - 1/h(k))/2 - (theta(k-1) + theta(k))/4 ],
//   rp[k] = rho0 cs2 [ (1/h(k+1) - 1/h(k))/2 + (theta(k+1) + theta(k))/4 ],
// and the MIE pull corrections (multiplied by B_rest and the other axis' h)
//   dm[k] = W1 (h(k-1) - h(k)) + csm2 (h^2 theta(k-1) + h^2 theta(k))/4,
//   dp[k] = W1 (h(k+1) - h(k)) - csm2 (h^2 theta(k+1) + h^2 theta(k))/4, W1 = csm2/2.
// Entries whose neighbour lies beyond a wall are never used (that link
// bounces back) and are set to 0.
__global__ void axis_tables_kernel(const double *h, const double *th, int n, int periodic,
                                   double rho0cs2, double csm2, float *out /* [7][n] */) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const bool has_m = periodic || k > 0, has_p = periodic || k < n - 1;
    const int km = periodic ? (k - 1 + n) % n : (k > 0 ? k - 1 : k);
    const int kp = periodic ? (k + 1) % n : (k < n - 1 ? k + 1 : k);
    out[0 * n + k] = (float)h[k];
    out[1 * n + k] = (float)(1.0 / h[k]);
    out[2 * n + k] = (float)th[k];
    out[3 * n + k] = has_m ? (float)(rho0cs2 * (0.5 * (1.0 / h[km] - 1.0 / h[k]) - 0.25 * (th[km] + th[k]))) : 0.f;
    out[4 * n + k] = has_p ? (float)(rho0cs2 * (0.5 * (1.0 / h[kp] - 1.0 / h[k]) + 0.25 * (th[kp] + th[k]))) : 0.f;
    const double W1 = 0.5 * csm2;
    const double ht = h[k] * h[k] * th[k], htm = h[km] * h[km] * th[km], htp = h[kp] * h[kp] * th[kp];
    out[5 * n + k] = has_m ? (float)(W1 * (h[km] - h[k]) + 0.25 * csm2 * (htm + ht)) : 0.f;
    out[6 * n + k] = has_p ? (float)(W1 * (h[kp] - h[k]) - 0.25 * csm2 * (htp + ht)) : 0.f;
}

// FP32 tables of the curvilinear column metric ([10][n], layout of Axis): h1,
// 1/h1, theta11, the full pull corrections of links 1 and 3,
//   rm[k] = f_ref+,1(k-1) - f_ref-,1(k) = rho0 cs2 (r(k-1) - r(k))/2 + (Fr(k-1) + Fr(k))/4,
//   rp[k] = f_ref+,3(k+1) - f_ref-,3(k) = rho0 cs2 (r(k+1) - r(k))/2 - (Fr(k+1) + Fr(k))/4,
// with r = h2/h1 and the rest-state force Fr = h2 (theta21 - theta11) rho0 cs2
// (Eq. bodyforce1 at U = 0), then h2, 1/h2, theta21 in the rows the MIE
// corrections take on straight grids ([8][n]).
// The xi1 axis has walls, so k - 1 / k + 1 beyond them are never pulled from.
__global__ void annulus_tables_kernel(const double *m, int n, double rho0cs2, float *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int w = n + 2;
    const double *h1 = m, *t11 = m + w, *h2 = m + 2 * w, *t21 = m + 3 * w;
    auto rr = [&](int q) { return h2[q] / h1[q]; };
    auto fr = [&](int q) { return h2[q] * (t21[q] - t11[q]) * rho0cs2; };
    out[0 * n + k] = (float)h1[k];
    out[1 * n + k] = (float)(1.0 / h1[k]);
    out[2 * n + k] = (float)t11[k];
    out[3 * n + k] = k > 0 ? (float)(0.5 * rho0cs2 * (rr(k - 1) - rr(k)) + 0.25 * (fr(k - 1) + fr(k))) : 0.f;
    out[4 * n + k] = k < n - 1 ? (float)(0.5 * rho0cs2 * (rr(k + 1) - rr(k)) - 0.25 * (fr(k + 1) + fr(k))) : 0.f;
    out[5 * n + k] = (float)h2[k];
    out[6 * n + k] = (float)(1.0 / h2[k]);
    out[7 * n + k] = (float)t21[k];
}

__global__ void fill_kernel(double *p, long long n, double v) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        p[k] = v;
}

// FP32 node-table metric for the step kernel (StepParams.gm) from the FP64
// table [6][ny][nx] (h1, h2, theta11, theta12, theta21, theta22): the six
// planes, then the full pull corrections of links 1..4 into each node,
//   link 1 (source i-1): rho0 cs2 (r(src) - r)/2 + (Fr1(src) + Fr1)/4,
//   link 3 (source i+1): rho0 cs2 (r(src) - r)/2 - (Fr1(src) + Fr1)/4,
//   link 2 (source j-1): rho0 cs2 (s(src) - s)/2 + (Fr2(src) + Fr2)/4,
//   link 4 (source j+1): rho0 cs2 (s(src) - s)/2 - (Fr2(src) + Fr2)/4,
// r = h2/h1, s = h1/h2, Fr = (h2 (theta21 - theta11), h1 (theta12 - theta22))
// rho0 cs2 (Eq. bodyforce1/2 at U = 0); 0 where the source lies beyond a wall.
__global__ void table_metric_kernel(const double *tab, int nx, int ny, int pitch, long long plane, int per_x,
                                    int per_y, double rho0cs2, float *gm) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= nx || j >= ny) return;
    const long long N = (long long)nx * ny;
    auto at = [&](int k, int ii, int jj) { return tab[k * N + (long long)jj * nx + ii]; };
    auto r_ = [&](int ii, int jj) { return at(1, ii, jj) / at(0, ii, jj); };
    auto s_ = [&](int ii, int jj) { return at(0, ii, jj) / at(1, ii, jj); };
    auto f1 = [&](int ii, int jj) { return at(1, ii, jj) * (at(4, ii, jj) - at(2, ii, jj)) * rho0cs2; };
    auto f2 = [&](int ii, int jj) { return at(0, ii, jj) * (at(3, ii, jj) - at(5, ii, jj)) * rho0cs2; };
    const long long o = (long long)j * pitch + i;
    for (int k = 0; k < 6; k++) gm[k * plane + o] = (float)at(k, i, j);
    const int im = per_x ? (i - 1 + nx) % nx : i - 1, ip = per_x ? (i + 1) % nx : i + 1;
    const int jm = per_y ? (j - 1 + ny) % ny : j - 1, jp = per_y ? (j + 1) % ny : j + 1;
    gm[6 * plane + o] = im >= 0 ? (float)(0.5 * rho0cs2 * (r_(im, j) - r_(i, j)) + 0.25 * (f1(im, j) + f1(i, j))) : 0.f;
    gm[7 * plane + o] = jm >= 0 ? (float)(0.5 * rho0cs2 * (s_(i, jm) - s_(i, j)) + 0.25 * (f2(i, jm) + f2(i, j))) : 0.f;
    gm[8 * plane + o] = ip < nx ? (float)(0.5 * rho0cs2 * (r_(ip, j) - r_(i, j)) - 0.25 * (f1(ip, j) + f1(i, j))) : 0.f;
    gm[9 * plane + o] = jp < ny ? (float)(0.5 * rho0cs2 * (s_(i, jp) - s_(i, j)) - 0.25 * (f2(i, jp) + f2(i, j))) : 0.f;
}

// ---- initial state (Appendix C.1): f = P^-1 m^eq,eff(rho, U), gradients by
// the same second-order differences as the step; g = g^eq(0) + g^corr.
// FP64 arithmetic (one-off).  Fields are [ny][nx] doubles on the device.
struct InitParams {
    StepParams sp;
    const double *h1d, *h2d, *t1d, *t2d;   // FP64 node metric per axis
    const double *h2x, *t21x;              // curvilinear column metric: h2, theta21 over xi1 (else null)
    double cs2, nu, zeta, rho0, csm2, eta;
    int gi, mhd;
    // the five fields rho, U1, U2, B1, B2 as [ny][nx] FP64 arrays; field k is
    // the constant cval[k] instead where bit k of cmask is set (no array)
    const double *rho, *u1, *u2, *b1, *b2;
    double cval[5];
    int cmask;
};

// field k of the initial state at node n
__device__ __forceinline__ double init_field(const InitParams &q, int k, long long n) {
    if (q.cmask >> k & 1) return q.cval[k];
    const double *a[5] = {q.rho, q.u1, q.u2, q.b1, q.b2};
    return a[k][n];
}

// second-order derivative of field k along an axis (central; one-sided at
// the first and last node of a wall axis)
__device__ double dfd64(const InitParams &q, int fk, int i, int j, int nx, int ny, int axis, int per) {
    auto at = [&](int ii, int jj) { return init_field(q, fk, (long long)jj * nx + ii); };
    const int k = axis == 0 ? i : j, n = axis == 0 ? nx : ny;
    auto nb = [&](int off) {
        int kk = k + off;
        if (per) kk = ((kk % n) + n) % n;
        return axis == 0 ? at(kk, j) : at(i, kk);
    };
    if (per || (k > 0 && k < n - 1)) return 0.5 * (nb(1) - nb(-1));
    if (k == 0) return 0.5 * (-3.0 * nb(0) + 4.0 * nb(1) - nb(2));
    return 0.5 * (3.0 * nb(0) - 4.0 * nb(-1) + nb(-2));
}

template <class S>
__global__ void init_kernel(const InitParams q) {
    const StepParams &p = q.sp;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= p.nx || j >= p.ny) return;
    const long long n = (long long)j * p.nx + i, idx = (long long)j * p.pitch + i;
    const bool curv = q.h2x != nullptr;
    double h1 = q.h1d[i], h2 = curv ? q.h2x[i] : q.h2d[j], t11 = q.t1d[i], t22 = curv ? 0.0 : q.t2d[j];
    double t21 = curv ? q.t21x[i] : 0.0, t12 = 0.0;
    if (p.curv == 2) {   // node table: the FP32 planes the step kernel uses
        h1 = gm_at(p.gm, p.plane, p.pitch, 0, i, j);
        h2 = gm_at(p.gm, p.plane, p.pitch, 1, i, j);
        t11 = gm_at(p.gm, p.plane, p.pitch, 2, i, j);
        t12 = gm_at(p.gm, p.plane, p.pitch, 3, i, j);
        t21 = gm_at(p.gm, p.plane, p.pitch, 4, i, j);
        t22 = gm_at(p.gm, p.plane, p.pitch, 5, i, j);
    }
    const double rho = init_field(q, 0, n), U1 = init_field(q, 1, n), U2 = init_field(q, 2, n);
    const double dU1 = dfd64(q, 1, i, j, p.nx, p.ny, 0, p.per_x);
    const double dU2 = dfd64(q, 2, i, j, p.nx, p.ny, 1, p.per_y);
    const double dr1 = dfd64(q, 0, i, j, p.nx, p.ny, 0, p.per_x);
    const double dr2 = dfd64(q, 0, i, j, p.nx, p.ny, 1, p.per_y);
    const double cs2 = q.cs2, nu = q.nu, ze = q.zeta;
    const double gi = q.gi ? 1.0 : 0.0;
    const double a1 = gi * U1 * U1 / cs2, a2 = gi * U2 * U2 / cs2;
    // Eqs. 83 / 85 (theta12, theta21 on curvilinear grids)
    const double tc11 = rho * (ze + nu) * U2 * t12 + rho * (ze - nu) * U1 * t21;   // Eq. tauc
    const double tc22 = rho * (ze + nu) * U1 * t21 + rho * (ze - nu) * U2 * t12;
    const double D31 = rho * (2 * ze - (ze + nu) * h2 / (h1 * h1) - (ze - nu) / h2
                              - ze * (2 - h2 / cs2 + (3 * a1 + 1) * h2 / (h1 * h1)));
    const double D32 = rho * (2 * ze - (ze + nu) * h1 / (h2 * h2) - (ze - nu) / h1
                              - ze * (2 - h1 / cs2 + (3 * a2 + 1) * h1 / (h2 * h2)));
    const double D33 = -ze * ((3 - a1) * h2 / (h1 * h1) - h2 / cs2 - a2 / h2) * U1;
    const double D34 = -ze * ((3 - a2) * h1 / (h2 * h2) - h1 / cs2 - a1 / h1) * U2;
    const double C3 = rho * ze * (2 * U1 * (a1 + 1) * h2 / h1 * t11 + 2 * U2 * (a2 + 1) * h1 / h2 * t22)
                      - (h2 / h1 * tc11 + h1 / h2 * tc22)
                      - rho * ze * U1 * ((3 + a1) * h2 / h1 + 2 * h1 / h2 - h1 * h2 / cs2) * t21
                      - rho * ze * U2 * ((3 + a2) * h1 / h2 + 2 * h2 / h1 - h1 * h2 / cs2) * t12;
    const double D41 = rho * (2 * nu - (ze + nu) * h2 / (h1 * h1) + (ze - nu) / h2
                              - nu * (2 - h2 / cs2 + (3 * a1 + 1) * h2 / (h1 * h1)));
    const double D42 = rho * (-2 * nu + (ze + nu) * h1 / (h2 * h2) - (ze - nu) / h1
                              - nu * (-2 + h1 / cs2 - (3 * a2 + 1) * h1 / (h2 * h2)));
    const double D43 = -nu * ((3 - a1) * h2 / (h1 * h1) - h2 / cs2 + a2 / h2) * U1;
    const double D44 = -nu * (-(3 - a2) * h1 / (h2 * h2) + h1 / cs2 - a1 / h1) * U2;
    const double C4 = rho * nu * (2 * U1 * (a1 + 1) * h2 / h1 * t11 - 2 * U2 * (a2 + 1) * h1 / h2 * t22)
                      - (h2 / h1 * tc11 - h1 / h2 * tc22)
                      - rho * nu * U1 * ((3 + a1) * h2 / h1 - 2 * h1 / h2 - h1 * h2 / cs2) * t21
                      - rho * nu * U2 * (-(3 + a2) * h1 / h2 + 2 * h2 / h1 + h1 * h2 / cs2) * t12;
    const double n3 = D31 * dU1 + D32 * dU2 + D33 * dr1 + D34 * dr2 + C3;
    const double n4 = D41 * dU1 + D42 * dU2 + D43 * dr1 + D44 * dr2 + C4;
    // m^eq,eff - m_rest(rho0), bare order (Eq. GOCmomentequilibria)
    const double r = h2 / h1, s = h1 / h2, H = h1 * h2;
    const double k2s = r * rho * U1 * U1 + s * rho * U2 * U2 + (r + s) * rho * cs2 + n3;
    const double k2d = r * rho * U1 * U1 - s * rho * U2 * U2 + (r - s) * rho * cs2 + n4;
    const double m0 = H * (rho - q.rho0);
    const double m1 = h2 * rho * U1, m2 = h1 * rho * U2;
    const double m3 = 0.5 * (k2s + k2d) - r * q.rho0 * cs2;
    const double m4 = 0.5 * (k2s - k2d) - s * q.rho0 * cs2;
    const double m5 = rho * U1 * U2;
    const double m6 = rho * (cs2 + U1 * U1) * U2 / h1;
    const double m7 = rho * (cs2 + U2 * U2) * U1 / h2;
    const double m8 = rho * cs2 * cs2 + rho * cs2 * (U1 * U1 + U2 * U2) + rho * U1 * U1 * U2 * U2
                      - q.rho0 * cs2 * cs2;
    double d[9];
    d[0] = m0 - m3 - m4 + m8;
    d[1] = 0.5 * (m1 + m3 - m7 - m8);
    d[2] = 0.5 * (m2 + m4 - m6 - m8);
    d[3] = 0.5 * (-m1 + m3 + m7 - m8);
    d[4] = 0.5 * (-m2 + m4 + m6 - m8);
    d[5] = 0.25 * (m5 + m6 + m7 + m8);
    d[6] = 0.25 * (-m5 + m6 - m7 + m8);
    d[7] = 0.25 * (m5 - m6 - m7 + m8);
    d[8] = 0.25 * (-m5 - m6 + m7 + m8);
    // pre-collision reference f_ref- = f_rest - F_rest/4 on links 1, 3 (xi1) and 2, 4 (xi2)
    const double F1r = h2 * q.rho0 * cs2 * (t21 - t11), F2r = h1 * q.rho0 * cs2 * (t12 - t22);
    d[1] += 0.25 * F1r;
    d[3] -= 0.25 * F1r;
    constexpr bool scaled = Store<S>::scaled;
    if (scaled && !p.curv) {   // per-row reference of 16-bit storage: +-u1r on links 1, 3
        d[1] -= (double)GOC_U1R(p, j);
        d[3] += (double)GOC_U1R(p, j);
    }
    d[2] += 0.25 * F2r;
    d[4] -= 0.25 * F2r;
    S *fout = static_cast<S *>(p.fout);
    for (int a = 0; a < 9; a++) Store<S>::st(fout + a * p.plane + idx, (float)(d[a] * p.isf));
    S *Fout = static_cast<S *>(p.Fout);   // F^{-1} = 0, i.e. F_dev = -F_rest
    Store<S>::st(Fout + idx, (float)(-F1r * p.isF));
    Store<S>::st(Fout + p.plane + idx, (float)(-F2r * p.isF));
    if (!q.mhd) return;
    S *gout = static_cast<S *>(p.gout);
    const double B[2] = {init_field(q, 3, n), init_field(q, 4, n)}, U[2] = {U1, U2};
    for (int c = 0; c < 2; c++) {
        const double dB1 = dfd64(q, 3 + c, i, j, p.nx, p.ny, 0, p.per_x);
        const double dB2 = dfd64(q, 3 + c, i, j, p.nx, p.ny, 1, p.per_y);
        const double A1 = U1 * B[c] - B[0] * U[c], A2 = U2 * B[c] - B[1] * U[c];
        // Eq. 42_C (theta21, theta12 on curvilinear grids)
        const double lc1 = q.eta * (H - h2 / h1) * dB1 + q.eta * h1 * H * (t11 + t21) * B[c];
        const double lc2 = q.eta * (H - h1 / h2) * dB2 + q.eta * H * h2 * (t22 + t12) * B[c];
        // relative to the pre-collision reference g_ref- = W H B_rest - e.M/2 with
        // M = csm2/2 (h1 H theta11, H h2 theta22) B_rest (B_rest = 0 on curvilinear grids)
        const double br = (scaled && !p.curv) ? (double)bref<true>(p, c, j) : (double)p.brest[c];
        const double M1 = 0.5 * q.csm2 * h1 * H * t11 * br, M2 = 0.5 * q.csm2 * H * h2 * t22 * br;
        for (int a = 0; a < 5; a++) {
            const double W = a == 0 ? 1.0 - 2.0 * q.csm2 : 0.5 * q.csm2;
            const double geq = W * (H * (B[c] - br) + g1(a) * (h2 * A1 + lc1) / q.csm2
                                    + g2(a) * (h1 * A2 + lc2) / q.csm2)
                               + 0.5 * (g1(a) * M1 + g2(a) * M2);
            Store<S>::st(gout + (c * 5 + a) * p.plane + idx, (float)(geq * p.isg));
        }
    }
}

// ---- macroscopic fields of the current state (FP64 output [5][ny][nx]) ----
template <class S, bool MHD>
__global__ void moments_kernel(const StepParams p, double *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= p.nx || j >= p.ny) return;
    const SrcGlobal<S> src{static_cast<const S *>(p.fin), static_cast<const S *>(p.Fin), static_cast<const S *>(p.gin),
                           p.plane, p.pitch, p.sf, p.sF, p.sg};
    constexpr bool REF = Store<S>::scaled;   // 16-bit storage: straight grids carry the per-row reference
    float h1, h2, ih1, ih2;
    float d[9];
    float ur1 = 0.f;
    if (p.curv == 2) {
        node_metric<2>(p, i, j, h1, h2, ih1, ih2);
        pull_node<true, 2>(p, src, i, j, h1, h2, d);
    } else if (p.curv) {
        node_metric<1>(p, i, j, h1, h2, ih1, ih2);
        pull_node<true, 1>(p, src, i, j, h1, h2, d);
    } else {
        node_metric<0>(p, i, j, h1, h2, ih1, ih2);
        if (REF) ur1 = GOC_U1R(p, j);
        pull_node<true, 0, REF>(p, src, i, j, h1, h2, d, ur1);
    }
    float drho, U1, U2;
    // F - F_rest of the previous step (the body force, or zero before the first step, without a stored force)
    const float F1p = p.constF ? (p.nopull ? 0.f : p.fext1) : src.Fv(0, i, j);
    const float F2p = p.constF ? (p.nopull ? 0.f : p.fext2) : src.Fv(1, i, j);
    fields_from<REF>(p, d, F1p, F2p, ih1, ih2, drho, U1, U2, ur1);
    const long long N = (long long)p.nx * p.ny, n = (long long)j * p.nx + i;
    out[n] = (double)p.rho0 + (double)drho;
    out[N + n] = U1;
    out[2 * N + n] = U2;
    double B1 = 0.0, B2 = 0.0;
    if constexpr (MHD) {
        float gd[2][5];
        for (int c = 0; c < 2; c++) {
            if (p.curv == 2) pull_mie<true, 2>(p, src, i, j, h1, h2, c, gd[c]);
            else if (p.curv) pull_mie<true, 1>(p, src, i, j, h1, h2, c, gd[c]);
            else pull_mie<true, 0, REF>(p, src, i, j, h1, h2, c, gd[c]);
        }
        const float s0 = (gd[0][0] + gd[0][1] + gd[0][2] + gd[0][3] + gd[0][4]) / (h1 * h2);
        const float s1 = (gd[1][0] + gd[1][1] + gd[1][2] + gd[1][3] + gd[1][4]) / (h1 * h2);
        if (p.curv) {   // h1 h2 B = sum g - Y/2 (Eq. 13_C, Eq. 6ab_C), as in the step kernel
            const float t12 = p.curv == 2 ? gm_at(p.gm, p.plane, p.pitch, 3, i, j) : 0.f;
            const float t21 = p.curv == 2 ? gm_at(p.gm, p.plane, p.pitch, 4, i, j) : curv_t21(p.ax1, p.nx, i);
            const float a11 = 1.f + 0.5f * t12 * U2, a12 = -0.5f * t12 * U1;
            const float a21 = -0.5f * t21 * U2, a22 = 1.f + 0.5f * t21 * U1;
            const float det = a11 * a22 - a12 * a21;
            B1 = (double)((s0 * a22 - a12 * s1) / det);
            B2 = (double)((a11 * s1 - a21 * s0) / det);
        } else {
            B1 = (double)bref<REF>(p, 0, j) + (double)s0;
            B2 = (double)bref<REF>(p, 1, j) + (double)s1;
        }
    }
    out[3 * N + n] = B1;
    out[4 * N + n] = B2;
}

// ---- per-row storage reference of 16-bit storage on straight grids ----------
// The stored deviations of links 1 and 3 are relative to a reference carrying
// the momentum h2 rho0 A1(j) of a row velocity A1(j); the MIE populations are
// relative to g_ref = W H Bref(j) -+ e.M/2 with a row field Bref_c(j) (M as for
// B_rest).  A refresh sets A1 and Bref to the row means of U1 and B of the
// current state (ref_rows_kernel), re-expresses the stored values against the
// new reference (ref_apply_kernel), then rebuilds the FP32 tables
// (ref_tables_kernel).  The FP64 master rows ref[3][ny] are A1, Bref_1, Bref_2.

// u1r of row j: the value the step kernel reads, from the FP64 master rows
__device__ __forceinline__ float ref_u1r(const double *h2, const double *ref, double rho0, int j) {
    return (float)(0.5 * rho0 * h2[j] * ref[j]);
}

// FP32 tables u1r [ny], brow [2][ny], bpull [4][ny] (links 2 and 4, per unit
// h1: g_ref+(source row) - g_ref-(row j), the MIE analogue of the f_ref
// corrections; 0 where the source row lies beyond a wall)
__global__ void ref_tables_kernel(const double *h2, const double *t2, int ny, int per_y, double rho0, double csm2,
                                  const double *ref, float *u1r, float *brow, float *bpull) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ny) return;
    u1r[j] = ref_u1r(h2, ref, rho0, j);
    const bool has_m = per_y || j > 0, has_p = per_y || j < ny - 1;
    const int jm = per_y ? (j - 1 + ny) % ny : (j > 0 ? j - 1 : j);
    const int jp = per_y ? (j + 1) % ny : (j < ny - 1 ? j + 1 : j);
    const double W1 = 0.5 * csm2;
    for (int c = 0; c < 2; c++) {
        const double *B = ref + (1 + c) * ny;
        brow[c * ny + j] = (float)B[j];
        const double hb = h2[j] * B[j], hm = h2[jm] * B[jm], hp = h2[jp] * B[jp];
        const double tb = h2[j] * h2[j] * t2[j] * B[j], tm = h2[jm] * h2[jm] * t2[jm] * B[jm],
                     tp = h2[jp] * h2[jp] * t2[jp] * B[jp];
        bpull[c * ny + j] = has_m ? (float)(W1 * (hm - hb) + 0.25 * csm2 * (tm + tb)) : 0.f;
        bpull[(2 + c) * ny + j] = has_p ? (float)(W1 * (hp - hb) - 0.25 * csm2 * (tp + tb)) : 0.f;
    }
}

// Row means of U1 and B of the current state, one block of 256 threads per
// row, summed in a fixed order (the refresh is reproducible): out[3][ny].
// Each node's values come from its own stored populations and force only (no
// pulls), so a slab's rows next to a cut need no fresh ghost rows: after a
// step the stored post-collision populations hold the momentum h2 rho U1 +
// F1/2 (exactly with omega1 = 1; the reference only has to be close to the
// flow), i.e. U1 = (sum d e1 + 2 u1r - (F1 - F1_rest)/2) / (rho h2), and the
// MIE zeroth moment h1 h2 (B - Bref) = sum g (Y = 0 on straight grids); the
// initial pre-collision state (pre = 1) gives U1 by Eq.
// GOChydrodynamicfields, with + (F1 - F1_rest)/2.
// lay: where the populations sit (AA_C for two-buffer lattices; an in-place
// lattice's layout, goc_aa.cuh)
template <class S, bool MHD>
__global__ void ref_rows_kernel(const StepParams p, double *out, int pre, int lay) {
    static_assert(Store<S>::scaled, "the per-row reference belongs to 16-bit storage");
    __shared__ double red[3][256];
    const int j = blockIdx.x, t = threadIdx.x;
    const S *fb = static_cast<const S *>(p.fin), *gb = static_cast<const S *>(p.gin);
    double acc[3] = {0.0, 0.0, 0.0};
    const float fs = pre ? 0.5f : -0.5f;
    for (int i = t; i < p.nx; i += 256) {
        float h1, h2, ih1, ih2, d[9];
        node_metric<0>(p, i, j, h1, h2, ih1, ih2);
#pragma unroll
        for (int a = 0; a < 9; a++) d[a] = scl<S>(Store<S>::ld(fb + aa_slot(p, lay, a, i, j)), p.sf);
        float k00 = 0.f;
#pragma unroll
        for (int a = 0; a < 9; a++) k00 += d[a];
        const float k10 = d[1] - d[3] + d[5] - d[6] - d[7] + d[8];
        const float rho = p.rho0 + k00 * (ih1 * ih2);
        const float F1 = scl<S>(Store<S>::ld(static_cast<const S *>(p.Fin) + (long long)j * p.pitch + i), p.sF);
        const float U1 = (k10 + fmaf(fs, F1, 2.f * GOC_U1R(p, j))) / rho * ih2;
        acc[0] += (double)U1;
        if constexpr (MHD) {
            for (int c = 0; c < 2; c++) {
                float sum = 0.f;
                for (int a = 0; a < 5; a++) sum += scl<S>(Store<S>::ld(gb + aa_slot(p, lay, a, i, j, true, c)), p.sg);
                acc[1 + c] += (double)GOC_BROW(p, c, j) + (double)(sum * (ih1 * ih2));
            }
        }
    }
    for (int k = 0; k < 3; k++) red[k][t] = acc[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (t < w)
            for (int k = 0; k < 3; k++) red[k][t] += red[k][t + w];
        __syncthreads();
    }
    if (t == 0) {
        out[j] = red[0][0] / p.nx;
        out[p.ny + j] = MHD ? red[1][0] / p.nx : (double)p.brest[0];
        out[2 * p.ny + j] = MHD ? red[2][0] / p.nx : (double)p.brest[1];
    }
}

// Re-express the stored values of the current buffer (post-collision, or the
// pre-collision f^0 when pre = 1) against the new reference rows refn: the
// stored value plus f_ref(old) - f_ref(new), rounded like every stored value
// (stochastically unless round-to-nearest storage was asked for).  The old
// reference is read from the tables the step kernel uses (p.u1r, p.brow).
template <class S, bool MHD>
__global__ void ref_apply_kernel(const StepParams p, const double *h1d, const double *t1d, const double *h2d,
                                 const double *t2d, const double *refn, double rho0, double csm2, int pre,
                                 unsigned salt, int lay) {
    static_assert(Store<S>::scaled, "the per-row reference belongs to 16-bit storage");
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= p.nx || j >= p.ny) return;
    const long long idx = (long long)j * p.pitch + i;
    uint32_t rng = node_seed((uint32_t)(idx + (long long)p.seed_row0 * p.pitch), salt);
    const bool sr = p.sr != 0;
    S *f = static_cast<S *>(const_cast<void *>(p.fin));
    const double du = (double)GOC_U1R(p, j) - (double)ref_u1r(h2d, refn, rho0, j);
    if (du != 0.0) {
        S *f1 = f + aa_slot(p, lay, 1, i, j), *f3 = f + aa_slot(p, lay, 3, i, j);
        const double v1 = (double)Store<S>::ld(f1) * p.sf + du, v3 = (double)Store<S>::ld(f3) * p.sf - du;
        put<S>(f1, (float)(v1 * p.isf), sr, rng);
        put<S>(f3, (float)(v3 * p.isf), sr, rng);
    }
    if constexpr (MHD) {
        S *g = static_cast<S *>(const_cast<void *>(p.gin));
        const double H = h1d[i] * h2d[j], sgn = pre ? -1.0 : 1.0;
        for (int c = 0; c < 2; c++) {
            const double dB = (double)GOC_BROW(p, c, j) - (double)(float)refn[(1 + c) * p.ny + j];
            if (dB == 0.0) continue;
            const double M1 = 0.5 * csm2 * dB * h1d[i] * H * t1d[i], M2 = 0.5 * csm2 * dB * H * h2d[j] * t2d[j];
            for (int a = 0; a < 5; a++) {
                const double W = a == 0 ? 1.0 - 2.0 * csm2 : 0.5 * csm2;
                const double shift = W * H * dB + sgn * 0.5 * (g1(a) * M1 + g2(a) * M2);
                S *ga = g + aa_slot(p, lay, a, i, j, true, c);
                put<S>(ga, (float)(((double)Store<S>::ld(ga) * p.sg + shift) * p.isg), sr, rng);
            }
        }
    }
}

// ---- FP64 reductions ---------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int K>
__device__ void block_add(double (&v)[K], double *dst) {
    __shared__ double red[K][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; k++) {
        double s = warp_sum(v[k]);
        if (lane == 0) red[k][w] = s;
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            double s = lane < (int)(blockDim.x >> 5) ? red[k][lane] : 0.0;
            s = warp_sum(s);
            if (lane == 0) atomicAdd(dst + k, s);
        }
    }
}

// h1 h2 of node (i, j) in FP64 for every grid kind: per-axis tables
// (straight), the column metric (annular sector: h2 a function of xi1) or the
// node table.  The rest-state mass of the node is this times rho0.
__device__ __forceinline__ double node_h1h2(const StepParams &p, int i, int j) {
    if (p.curv == 2) return (double)gm_at(p.gm, p.plane, p.pitch, 0, i, j) * gm_at(p.gm, p.plane, p.pitch, 1, i, j);
    return (double)p.ax1.h[i] * (double)(p.curv ? curv_h2(p.ax1, i) : p.ax2.h[j]);
}

// Total mass sum_nodes sum_a f (= sum h1 h2 rho): post-collision deviations
// plus h1 h2 rho0 per node (mass is a collision invariant).
template <class S>
__global__ void mass_kernel(const StepParams p, double *out) {
    double acc[1] = {0.0};
    const long long N = (long long)p.nx * (p.own1 - p.own0);   // the owned rows
    const S *f = static_cast<const S *>(p.fin);
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const int j = p.own0 + (int)(n / p.nx), i = (int)(n - (long long)(j - p.own0) * p.nx);
        const long long idx = (long long)j * p.pitch + i;
        double s = 0.0;
        for (int a = 0; a < 9; a++) s += (double)Store<S>::ld(f + a * p.plane + idx) * p.sf;
        acc[0] += s + node_h1h2(p, i, j) * p.rho0;
    }
    block_add<1>(acc, out);
}

// Residual sums between two field snapshots [4][plane]: |dU|^2, |U|^2, |dB|^2, |B|^2.
__global__ void residual_kernel(const float *a, const float *b, long long plane, int nx, int ny,
                                int pitch, double *out) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const long long N = (long long)nx * ny;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(n / nx), i = (int)(n - (long long)j * nx);
        const long long idx = (long long)j * pitch + i;
        const double u1 = b[idx], u2 = b[plane + idx], B1 = b[2 * plane + idx], B2 = b[3 * plane + idx];
        const double du1 = u1 - a[idx], du2 = u2 - a[plane + idx];
        const double dB1 = B1 - a[2 * plane + idx], dB2 = B2 - a[3 * plane + idx];
        acc[0] += du1 * du1 + du2 * du2;
        acc[1] += u1 * u1 + u2 * u2;
        acc[2] += dB1 * dB1 + dB2 * dB2;
        acc[3] += B1 * B1 + B2 * B2;
    }
    block_add<4>(acc, out);
}

// Per-index metric records of an axis from its table rows (h, ih, th, rm,
// rp, dm, dp of n values each), written after the table's 8 rows:
// rec[2k] = (h, ih, th, rm), rec[2k + 1] = (rp, dm, dp, 0).
__global__ void axis_records_kernel(float *tab, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float4 *rec = reinterpret_cast<float4 *>(tab + 8 * (size_t)n);
    rec[2 * k] = make_float4(tab[k], tab[n + k], tab[2 * n + k], tab[3 * n + k]);
    rec[2 * k + 1] = make_float4(tab[4 * n + k], tab[5 * n + k], tab[6 * n + k], 0.f);
}

}  // namespace goc
