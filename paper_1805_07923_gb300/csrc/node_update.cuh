// The per-coefficient SDC node update (Sec. 4.2, Eq.
// update_equation_sdcq_discrete_form; with tau the coarse-level form, Eq.
// modified_update_equation_sdcq_discrete_form), the implicit solve and
// F_I at the new node (Sec. 4.4), as device functions of the node kernels
// (sdc.cu, coriolis_implicit.cu) and the Coriolis term shared with the
// analysis kernels (rhs_kernels.cuh, legendre_tc.cu).  All float64.
#pragma once

#include <cuda_runtime.h>

namespace mlsdc {

constexpr int kMaxNodes = 9;

struct Phys {
    double inv_a2, phibar, nu;
};

// Row m+1 of the SDC matrices for one node update.
struct NodeRow {
    double qe[kMaxNodes], qi[kMaxNodes], q[kMaxNodes];
    double qimm;
    int m;    // updating node m+1
    int M;    // nodes 0..M
};

// The row with every coefficient multiplied by dt, formed on the host: the
// node kernels take it so that no thread repeats the uniform products (the
// same float64 products, so the results do not change).
__host__ __device__ inline NodeRow dt_scaled(NodeRow r, double dt) {
    for (int j = 0; j < kMaxNodes; ++j) {
        r.qe[j] *= dt;
        r.qi[j] *= dt;
        r.q[j] *= dt;
    }
    r.qimm *= dt;
    return r;
}

__device__ __forceinline__ double2 cax(double2 acc, double s, double2 x) {
    return make_double2(fma(s, x.x, acc.x), fma(s, x.y, acc.y));
}

// F_I = [ -Phibar delta + nu L Phi', nu L zeta, -L Phi' + nu L delta ], L = -n(n+1)/a^2
__device__ __forceinline__ void implicit_rhs_coef(double L, const Phys& ph, double2 p, double2 z, double2 d,
                                                  double2& fp, double2& fz, double2& fd) {
    const double nl = ph.nu * L;
    fp = make_double2(-ph.phibar * d.x + nl * p.x, -ph.phibar * d.y + nl * p.y);
    fz = make_double2(nl * z.x, nl * z.y);
    fd = make_double2(-L * p.x + nl * d.x, -L * p.y + nl * d.y);
}

// x - alpha F_I(x) = b, diagonal per coefficient (Sec. 4.4).
__device__ __forceinline__ void implicit_solve_coef(double L, double alpha, const Phys& ph, double2 bp,
                                                    double2 bz, double2 bd, double2& p, double2& z,
                                                    double2& d) {
    const double c = 1.0 - alpha * ph.nu * L;
    const double ic = 1.0 / c;
    const double den = 1.0 / (c * c - alpha * alpha * ph.phibar * L);
    z = make_double2(bz.x * ic, bz.y * ic);
    p = make_double2((c * bp.x - alpha * ph.phibar * bd.x) * den, (c * bp.y - alpha * ph.phibar * bd.y) * den);
    d = make_double2((bd.x - alpha * L * p.x) * ic, (bd.y - alpha * L * p.y) * ic);
}

// The two reciprocals of the solve, per degree n: with c = 1 - alpha nu L,
// (1/c, 1 / (c^2 - alpha^2 Phibar L)).  They depend only on the degree and on
// alpha = dt q~I_{m+1,m+1}, so a step computes them once per level and node
// (k_solve_coefs) instead of per coefficient and update.
__device__ __forceinline__ double2 solve_recips(double L, double alpha, const Phys& ph) {
    const double c = 1.0 - alpha * ph.nu * L;
    return make_double2(1.0 / c, 1.0 / (c * c - alpha * alpha * ph.phibar * L));
}

// implicit_solve_coef with the reciprocals r = solve_recips(L, alpha, ph).
__device__ __forceinline__ void implicit_solve_tab(double L, double alpha, const Phys& ph, double2 r, double2 bp,
                                                   double2 bz, double2 bd, double2& p, double2& z, double2& d) {
    const double c = 1.0 - alpha * ph.nu * L;
    const double ic = r.x, den = r.y;
    z = make_double2(bz.x * ic, bz.y * ic);
    p = make_double2((c * bp.x - alpha * ph.phibar * bd.x) * den, (c * bp.y - alpha * ph.phibar * bd.y) * den);
    d = make_double2((bd.x - alpha * L * p.x) * ic, (bd.y - alpha * L * p.y) * ic);
}

// Field f (0 Phi', 1 zeta, 2 delta) of implicit_solve_tab followed by
// implicit_rhs_coef: the new value th and its F_I, by the same expressions,
// without the other fields' work (zeta needs only its own right-hand side;
// Phi' and delta need both p and d).
__device__ __forceinline__ void node_solve_field(int f, double L, double alpha, const Phys& ph, double2 r,
                                                 double2 bp, double2 bz, double2 bd, double2& th, double2& fi) {
    const double ic = r.x, den = r.y;
    const double nl = ph.nu * L;
    if (f == 1) {
        th = make_double2(bz.x * ic, bz.y * ic);
        fi = make_double2(nl * th.x, nl * th.y);
        return;
    }
    const double c = 1.0 - alpha * ph.nu * L;
    const double2 p = make_double2((c * bp.x - alpha * ph.phibar * bd.x) * den, (c * bp.y - alpha * ph.phibar * bd.y) * den);
    const double2 d = make_double2((bd.x - alpha * L * p.x) * ic, (bd.y - alpha * L * p.y) * ic);
    if (f == 0) {
        th = p;
        fi = make_double2(-ph.phibar * d.x + nl * p.x, -ph.phibar * d.y + nl * p.y);
    } else {
        th = d;
        fi = make_double2(-L * p.x + nl * d.x, -L * p.y + nl * d.y);
    }
}

// The Coriolis (linear) part L_F of the right-hand side at coefficient (m, n), exactly, in
// float64 spectral arithmetic.  With f = 2 Omega mu, -div(f V) and curl(f V)
// are tridiagonal in n for each m:
//   dzeta  = -2 Omega (mu delta)_n - (2 Omega / a^2) [ i m psi_n + (H chi)_n ]
//   ddelta =  2 Omega (mu zeta)_n  - (2 Omega / a^2) [ i m chi_n - (H psi)_n ]
//   (mu x)_n = eps_n x_{n-1} + eps_{n+1} x_{n+1},
//   (H x)_n  = -(n-1) eps_n x_{n-1} + (n+2) eps_{n+1} x_{n+1},
// from mu P_n = eps_{n+1} P_{n+1} + eps_n P_{n-1} and H_n = (1 - mu^2) dP_n/dmu,
// projected on n <= R; psi, chi = -a^2/(n(n+1)) (zeta, delta).  Collecting
// the factors of each neighbour (the a^2 of psi, chi cancels the 1/a^2):
//   dzeta  = -2 Omega [ alpha delta_{n-1} + beta delta_{n+1} + gamma i zeta_n ]
//   ddelta =  2 Omega [ alpha zeta_{n-1}  + beta zeta_{n+1}  - gamma i delta_n ]
// with the plan's per-coefficient factors cor[4 idx .. +2] = (alpha, beta,
// gamma): 16 float64 operations per coefficient (float64 runs at a small
// fraction of the float32 rate on this GPU).  The mixed-precision paths add
// this term in float64 and send only the nonlinear part of the products
// through the reduced-precision transforms; the implicit-Coriolis splitting
// (coriolis_implicit.cu) adds it to F_I instead.  Adds dzeta to f1 and ddelta to f2.
// coriolis_terms takes the neighbours' values (zero outside m <= n <= R);
// coriolis_add reads them from a state [3][nc] in global memory.
// The vorticity row alone (needs delta_{n-1}, zeta_n, delta_{n+1}) and the
// divergence row alone (zeta_{n-1}, delta_n, zeta_{n+1}).
__device__ __forceinline__ void coriolis_zeta_row(const double* __restrict__ cf, double2 dl, double2 zk, double2 du,
                                                  double two_omega, double2& f1) {
    const double2 ab = *reinterpret_cast<const double2*>(cf);
    const double al = ab.x, be = ab.y, ga = cf[2];
    const double ux = fma(al, dl.x, fma(be, du.x, -ga * zk.y)), uy = fma(al, dl.y, fma(be, du.y, ga * zk.x));
    f1.x = fma(-two_omega, ux, f1.x);
    f1.y = fma(-two_omega, uy, f1.y);
}
__device__ __forceinline__ void coriolis_delta_row(const double* __restrict__ cf, double2 zl, double2 dk, double2 zu,
                                                   double two_omega, double2& f2) {
    const double2 ab = *reinterpret_cast<const double2*>(cf);
    const double al = ab.x, be = ab.y, ga = cf[2];
    const double vx = fma(al, zl.x, fma(be, zu.x, ga * dk.y)), vy = fma(al, zl.y, fma(be, zu.y, -ga * dk.x));
    f2.x = fma(two_omega, vx, f2.x);
    f2.y = fma(two_omega, vy, f2.y);
}
__device__ __forceinline__ void coriolis_terms(const double* __restrict__ cf, double2 zl, double2 zk, double2 zu,
                                               double2 dl, double2 dk, double2 du, double two_omega, double2& f1,
                                               double2& f2) {
    coriolis_zeta_row(cf, dl, zk, du, two_omega, f1);
    coriolis_delta_row(cf, zl, dk, zu, two_omega, f2);
}

// The operands of coriolis_add for one coefficient, read ahead of their use
// (the analysis epilogues issue these loads before they wait for their sums).
struct CorIn {
    double2 zl, zk, zu, dl, dk, du;
    double al, be, ga;
};
__device__ __forceinline__ CorIn coriolis_load(const double2* __restrict__ state, const double* __restrict__ cor,
                                               int nc, int R, int m, int n, int off) {
    const int k = n - m;
    const double2* z = state + nc + off;
    const double2* d = state + 2 * nc + off;
    CorIn c;
    c.zl = c.zu = c.dl = c.du = make_double2(0.0, 0.0);
    if (n - 1 >= m) { c.zl = z[k - 1]; c.dl = d[k - 1]; }
    if (n + 1 <= R) { c.zu = z[k + 1]; c.du = d[k + 1]; }
    c.zk = z[k];
    c.dk = d[k];
    const double* cf = cor + 4 * (size_t)(off + k);
    const double2 ab = *reinterpret_cast<const double2*>(cf);
    c.al = ab.x;
    c.be = ab.y;
    c.ga = cf[2];
    return c;
}
// coriolis_terms on loaded operands (the same operations in the same order).
__device__ __forceinline__ void coriolis_apply(const CorIn& c, double two_omega, double2& f1, double2& f2) {
    const double ux = fma(c.al, c.dl.x, fma(c.be, c.du.x, -c.ga * c.zk.y));
    const double uy = fma(c.al, c.dl.y, fma(c.be, c.du.y, c.ga * c.zk.x));
    f1.x = fma(-two_omega, ux, f1.x);
    f1.y = fma(-two_omega, uy, f1.y);
    const double vx = fma(c.al, c.zl.x, fma(c.be, c.zu.x, c.ga * c.dk.y));
    const double vy = fma(c.al, c.zl.y, fma(c.be, c.zu.y, -c.ga * c.dk.x));
    f2.x = fma(two_omega, vx, f2.x);
    f2.y = fma(two_omega, vy, f2.y);
}

__device__ inline void coriolis_add(const double2* __restrict__ state, const double* __restrict__ cor, int nc, int R,
                                    int m, int n, int off, double two_omega, double2& f1, double2& f2) {
    const int k = n - m;
    const double2* z = state + nc + off;
    const double2* d = state + 2 * nc + off;
    double2 zl{0, 0}, zu{0, 0}, dl{0, 0}, du{0, 0};
    if (n - 1 >= m) { zl = z[k - 1]; dl = d[k - 1]; }
    if (n + 1 <= R) { zu = z[k + 1]; du = d[k + 1]; }
    coriolis_terms(cor + 4 * (size_t)(off + k), zl, z[k], zu, dl, d[k], du, two_omega, f1, f2);
}

// The right-hand side b of the node update at one (field, coefficient)
// offset o of a member's node arrays ([M+1][3][nc], node = 3 nc):
//   b = Th[0] + sum_{j=1..m} dt (qE_j (FEn_j - FEo_j) + qI_j (FIn_j - FIo_j))
//       - dt qI_{m+1,m+1} FIo_{m+1} + sum_{j=0..M} dt q_j (FIo_j + FEo_j) [+ tau_{m+1}]
// `row` is dt_scaled.
__device__ __forceinline__ double2 node_rhs(const double2* Th, const double2* FIo, const double2* FEo,
                                            const double2* FIn, const double2* FEn, const double2* tau,
                                            size_t node, size_t o, const NodeRow& row) {
    const int m = row.m;
    double2 acc = Th[o];  // Theta^n (node 0)
    for (int j = 1; j <= m; ++j) {
        const size_t oj = j * node + o;
        const double2 de = make_double2(FEn[oj].x - FEo[oj].x, FEn[oj].y - FEo[oj].y);
        const double2 di = make_double2(FIn[oj].x - FIo[oj].x, FIn[oj].y - FIo[oj].y);
        acc = cax(acc, row.qe[j], de);
        acc = cax(acc, row.qi[j], di);
    }
    acc = cax(acc, -row.qimm, FIo[(m + 1) * node + o]);
    for (int j = 0; j <= row.M; ++j) {
        const size_t oj = j * node + o;
        const double2 s = make_double2(FIo[oj].x + FEo[oj].x, FIo[oj].y + FEo[oj].y);
        acc = cax(acc, row.q[j], s);
    }
    if (tau) {
        const double2 t = tau[(m + 1) * node + o];
        acc = make_double2(acc.x + t.x, acc.y + t.y);
    }
    return acc;
}

}  // namespace mlsdc
