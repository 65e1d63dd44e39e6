// dynamics.cuh -- device code of the abstraction builder (Sec. V-B): the
// box over-approximation of the attainable set of one cell under one input,
// quantised to an integer cell range.  Included by the builder kernels and by
// the recompute-mode relaxation so both produce bit-identical boxes (every
// translation unit is compiled with --fmad=false, so no expression below is
// contracted into an FMA).
//
// Systems (Eq. ode):
//   LINEAR2D    x0' = x1, x1' = u0.  The flow is linear, so the image of a
//               cell is the hull of its 4 corner images:
//               (x0 + tau x1 + tau^2/2 u0, x1 + tau u0).
//   UNICYCLE3D  x' = v cos th, y' = v sin th, th' = w, u = (v, w).
//   FIRE4D      x' = V cos psi + wind, y' = V sin psi, psi' = (g / V) tan phi,
//               V' = a, u = (phi, a).
// For the last two the box is c(tau) +- r(tau): c from the cell centre under
// x' = f(x,u), r from r(0) = eta/2 under r' = L r + w (growth bound; L bounds
// |df_i/dx_j| off the diagonal, w the disturbance), both with the classical
// RK4 scheme over `substeps` equal steps.
#pragma once
#include "bf_internal.cuh"

namespace bfk {

template <int D>
__device__ __forceinline__ void dyn_rhs(const DynDesc& dd, const double* x, const double* u, double* f) {
    if constexpr (D == 3) {
        f[0] = u[0] * cos(x[2]);
        f[1] = u[0] * sin(x[2]);
        f[2] = u[1];
    } else if constexpr (D == 4) {
        f[0] = x[3] * cos(x[2]) + dd.p[0];
        f[1] = x[3] * sin(x[2]);
        f[2] = (dd.p[1] / x[3]) * tan(u[0]);
        f[3] = u[1];
    }
}

// Growth-bound matrix L (row-major) and disturbance w.
template <int D>
__device__ __forceinline__ void dyn_growth(const DynDesc& dd, const double* u, double* L, double* w) {
#pragma unroll
    for (int i = 0; i < D * D; ++i) L[i] = 0.0;
    if constexpr (D == 3) {
        const double v = fabs(u[0]);
        L[0 * 3 + 2] = v;
        L[1 * 3 + 2] = v;
        w[0] = dd.p[0]; w[1] = dd.p[0]; w[2] = dd.p[0];
    } else if constexpr (D == 4) {
        const double vhi = dd.p[3], vlo = dd.p[2];
        L[0 * 4 + 2] = vhi; L[0 * 4 + 3] = 1.0;
        L[1 * 4 + 2] = vhi; L[1 * 4 + 3] = 1.0;
        L[2 * 4 + 3] = (dd.p[1] * tan(fabs(u[0]))) / (vlo * vlo);
        w[0] = dd.p[4]; w[1] = dd.p[4]; w[2] = dd.p[4]; w[3] = dd.p[4];
    }
}

template <int D>
__device__ __forceinline__ void growth_rhs(const double* L, const double* w, const double* r, double* q) {
#pragma unroll
    for (int i = 0; i < D; ++i) {
        double s = w[i];
#pragma unroll
        for (int j = 0; j < D; ++j) s = s + L[i * D + j] * r[j];
        q[i] = s;
    }
}

// One RK4 substep of the centre c and the radius r; inc01 receives the
// increments added to c[0] and c[1] (the right-hand sides of the built-in
// systems do not read x[0] and x[1], so these increments depend only on
// c[2..] and the input).
template <int D>
__device__ __forceinline__ void rk4_step(const DynDesc& dd, const double* u, const double* L, const double* w,
                                         double h, double hh, double h6, double* c, double* r, double* inc01) {
    double k1[D], k2[D], k3[D], k4[D], t[D];
    double q1[D], q2[D], q3[D], q4[D], tr[D];
    dyn_rhs<D>(dd, c, u, k1);
    growth_rhs<D>(L, w, r, q1);
#pragma unroll
    for (int i = 0; i < D; ++i) { t[i] = c[i] + hh * k1[i]; tr[i] = r[i] + hh * q1[i]; }
    dyn_rhs<D>(dd, t, u, k2);
    growth_rhs<D>(L, w, tr, q2);
#pragma unroll
    for (int i = 0; i < D; ++i) { t[i] = c[i] + hh * k2[i]; tr[i] = r[i] + hh * q2[i]; }
    dyn_rhs<D>(dd, t, u, k3);
    growth_rhs<D>(L, w, tr, q3);
#pragma unroll
    for (int i = 0; i < D; ++i) { t[i] = c[i] + h * k3[i]; tr[i] = r[i] + h * q3[i]; }
    dyn_rhs<D>(dd, t, u, k4);
    growth_rhs<D>(L, w, tr, q4);
#pragma unroll
    for (int i = 0; i < D; ++i) {
        const double inc = h6 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
        if (i < 2) inc01[i] = inc;
        c[i] = c[i] + inc;
        r[i] = r[i] + h6 * (q1[i] + 2.0 * q2[i] + 2.0 * q3[i] + q4[i]);
    }
}

template <int D>
__device__ void rk4_centre_radius(const DynDesc& dd, const double* u, double* c, double* r) {
    double L[D * D], w[D];
    dyn_growth<D>(dd, u, L, w);
    const double h = dd.tau / (double)dd.substeps;
    const double hh = h * 0.5, h6 = h / 6.0;
#pragma unroll 1
    for (int s = 0; s < dd.substeps; ++s) {
        double inc01[2];
        rk4_step<D>(dd, u, L, w, h, hh, h6, c, r, inc01);
    }
}

// The part of rk4_centre_radius shared by all cells with the same coordinates
// on dims >= 2 (ckey = their centre there): the dim-0/1 increments of every
// substep, the final centre on dims >= 2 and the final radius.  A cell's
// centre on dim 0 or 1 is its start plus the increments, added in order.
// Table entry layout (kRkEntry doubles): inc[kRkMaxSub][2], cfinal[2],
// rfinal[4].
constexpr int kRkMaxSub = 8;
constexpr int kRkEntry = 2 * kRkMaxSub + 2 + 4;
template <int D>
__device__ void rk4_shared_part(const DynDesc& dd, const double* u, const double* ckey, double (*inc)[2],
                                double* cfinal, double* rfinal) {
    double L[D * D], w[D], c[D], r[D];
    dyn_growth<D>(dd, u, L, w);
    const double h = dd.tau / (double)dd.substeps;
    const double hh = h * 0.5, h6 = h / 6.0;
    c[0] = 0.0;
    c[1] = 0.0;
#pragma unroll
    for (int d = 2; d < D; ++d) c[d] = ckey[d - 2];
#pragma unroll
    for (int d = 0; d < D; ++d) r[d] = dd.eta[d] * 0.5;
#pragma unroll 1
    for (int s = 0; s < dd.substeps; ++s) rk4_step<D>(dd, u, L, w, h, hh, h6, c, r, inc[s]);
#pragma unroll
    for (int d = 2; d < D; ++d) cfinal[d - 2] = c[d];
#pragma unroll
    for (int d = 0; d < D; ++d) rfinal[d] = r[d];
}

// Cells meeting [a, b] on one dim (half-open cells); false = blocked.
__device__ __forceinline__ bool quantise_dim(double a, double b, double glo, double eta, int n,
                                             int periodic, int& lo, int& hi) {
    const double fa = floor((a - glo) / eta);
    const double fb = floor((b - glo) / eta);
    if (!(fa == fa) || !(fb == fb)) return false;
    if (!periodic) {
        if (fa < 0.0 || fb > (double)(n - 1)) return false;
        lo = (int)fa;
        hi = (int)fb;
        return true;
    }
    const double len = fb - fa + 1.0;
    if (len >= (double)n) { lo = 0; hi = n - 1; return true; }
    double m = fmod(fa, (double)n);
    if (m < 0.0) m += (double)n;
    lo = (int)m;
    hi = (int)m + (int)len - 1;
    return true;
}

template <int D>
__device__ __forceinline__ void quantise_box(const DynDesc& dd, const GridDesc& g, const double* a,
                                             const double* e, Box<D>& b) {
    bool ok = true;
#pragma unroll
    for (int d = 0; d < D; ++d)
        if (ok) ok = quantise_dim(a[d], e[d], dd.glo[d], dd.eta[d], g.n[d], g.periodic[d], b.lo[d], b.hi[d]);
    if (!ok) {
        b.lo[0] = kBlocked;
#pragma unroll
        for (int d = 1; d < D; ++d) b.lo[d] = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) b.hi[d] = 0;
    }
}

template <int D>
__device__ Box<D> make_box(const DynDesc& dd, const GridDesc& g, const double* __restrict__ inputs,
                           long long c, int ui) {
    Box<D> b;
    int k[4];
    cell_coords(g, c, k);
    const double* u = inputs + (long long)ui * dd.udim;
    double a[D], e[D];
    if constexpr (D == 2) {
        const double tt = 0.5 * dd.tau * dd.tau;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const double x0 = dd.glo[0] + (double)(k[0] + (q & 1)) * dd.eta[0];
            const double x1 = dd.glo[1] + (double)(k[1] + ((q >> 1) & 1)) * dd.eta[1];
            const double y0 = (x0 + dd.tau * x1) + tt * u[0];
            const double y1 = x1 + dd.tau * u[0];
            if (q == 0 || y0 < a[0]) a[0] = y0;
            if (q == 0 || y0 > e[0]) e[0] = y0;
            if (q == 0 || y1 < a[1]) a[1] = y1;
            if (q == 0 || y1 > e[1]) e[1] = y1;
        }
    } else if constexpr (D >= 3) {
        double cc[D], rr[D];
#pragma unroll
        for (int d = 0; d < D; ++d) {
            cc[d] = dd.glo[d] + ((double)k[d] + 0.5) * dd.eta[d];
            rr[d] = dd.eta[d] * 0.5;
        }
        rk4_centre_radius<D>(dd, u, cc, rr);
#pragma unroll
        for (int d = 0; d < D; ++d) { a[d] = cc[d] - rr[d]; e[d] = cc[d] + rr[d]; }
    } else {
        // D == 1 has no built-in system; callers supply boxes.
        b.lo[0] = kBlocked; b.hi[0] = 0;
        return b;
    }
    quantise_box<D>(dd, g, a, e, b);
    return b;
}

// Box of cell k from the shared part of its (key, input) trajectory: the same
// operations as make_box, in the same order.
template <int D>
__device__ Box<D> box_from_shared(const DynDesc& dd, const GridDesc& g, const int* k,
                                  const double* __restrict__ entry) {
    Box<D> b;
    double a[D], e[D], cc[2];
#pragma unroll
    for (int d = 0; d < 2; ++d) cc[d] = dd.glo[d] + ((double)k[d] + 0.5) * dd.eta[d];
#pragma unroll 1
    for (int s = 0; s < dd.substeps; ++s) {
        cc[0] = cc[0] + __ldg(entry + 2 * s);
        cc[1] = cc[1] + __ldg(entry + 2 * s + 1);
    }
    const double* cfinal = entry + 2 * kRkMaxSub;
    const double* rfinal = cfinal + 2;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const double c = d < 2 ? cc[d] : __ldg(cfinal + d - 2);
        const double r = __ldg(rfinal + d);
        a[d] = c - r;
        e[d] = c + r;
    }
    quantise_box<D>(dd, g, a, e, b);
    return b;
}

// Index of a cell's shared-RK4 key (its coordinates on dims >= 2).
template <int D>
__device__ __forceinline__ int rk_key(const GridDesc& g, const int* k) {
    return D >= 4 ? k[2] + g.n[2] * k[3] : k[2];
}

}  // namespace bfk
