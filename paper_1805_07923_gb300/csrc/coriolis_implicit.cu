// The implicit-Coriolis splitting: the alternative to Sec. 4.1's split of
// F = F_I + F_E in which the Coriolis part L_F is treated implicitly,
// F_I = L_G + L_F and F_E = N (the paper keeps L_F in F_E).  In spectral space
// L_F couples, for each zonal wavenumber m, degree n to n - 1 and n + 1 (the
// mu and (1 - mu^2) d/dmu recurrences of the Legendre functions, see
// coriolis_terms), so the implicit system of Sec. 4.4 (Eq. implicit_systems),
// x - alpha F_I(x) = b, is no longer diagonal.  Phi' couples only to delta at
// its own coefficient and is eliminated first; what remains for each m is two
// complex tridiagonal systems, the chains
//   zeta_m, delta_{m+1}, zeta_{m+2}, ...   and   delta_m, zeta_{m+1}, delta_{m+2}, ...
// (zeta_n couples to delta_{n-1}, delta_{n+1}; delta_n to zeta_{n-1}, zeta_{n+1}).
// With sigma = 2 Omega alpha, c_n = 1 - alpha nu L_n, L_n = -n(n+1)/a^2 and
// the Coriolis factors (al, be, ga) of coefficient (m, n):
//   zeta_n:  (c_n + i sigma ga) zeta_n + sigma al delta_{n-1} + sigma be delta_{n+1} = b_zeta
//   delta_n: (c_n - alpha^2 Phibar L_n / c_n + i sigma ga) delta_n - sigma al zeta_{n-1}
//            - sigma be zeta_{n+1} = b_delta - alpha L_n b_Phi / c_n
//   Phi'_n = (b_Phi - alpha Phibar delta_n) / c_n
// The chains are factored once per level, node and step size (k_cor_factor:
// the Thomas algorithm's elimination, sequential along each chain).  Every
// solve then runs the two substitutions, each a first-order linear
// recurrence, as a warp-wide scan of affine maps: one warp per chain, a
// contiguous segment of the chain per lane.  All float64.
#include "internal.h"
#include "sdc_internal.h"

namespace mlsdc {

constexpr int kCorThreads = 128;  // per wavenumber: warps 0 and 1 solve the two chains

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a b + c
__device__ __forceinline__ double2 zfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 zrecip(double2 w) {
    const double s = 1.0 / fma(w.x, w.x, w.y * w.y);
    return make_double2(w.x * s, -w.y * s);
}
__device__ __forceinline__ double2 zneg(double2 a) { return make_double2(-a.x, -a.y); }
__device__ __forceinline__ double2 zshfl_up(double2 v, int d) {
    return make_double2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ double2 zshfl_down(double2 v, int d) {
    return make_double2(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d));
}

// z_k = p_k + q_k z_{k-1} for k = 0..n-1 with z_{-1} = 0 (Fwd), or
// z_k = p_k + q_k z_{k+1} for k = n-1..0 with z_n = 0 (!Fwd), over one warp.
// Lane l takes the segment [l s, l s + s), s = ceil(n / 32): it composes its
// elements' affine maps z -> p + q z, an inclusive warp scan composes the
// segments (ascending lanes for Fwd, descending otherwise), and the lane then
// runs its segment from the value the scan hands it.  pq(k, p, q) gives the
// coefficients (called twice per k), put(k, z) receives the result.
template <bool Fwd, class PQ, class Put>
__device__ __forceinline__ void warp_recurrence(int n, int lane, PQ pq, Put put) {
    const int s = (n + 31) >> 5;
    const int k0 = min(n, lane * s), k1 = min(n, k0 + s);
    double2 A = make_double2(1.0, 0.0), B = make_double2(0.0, 0.0);
    for (int i = 0; i < k1 - k0; ++i) {
        const int k = Fwd ? k0 + i : k1 - 1 - i;
        double2 p, q;
        pq(k, p, q);
        B = zfma(q, B, p);
        A = zmul(q, A);
    }
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const double2 A1 = Fwd ? zshfl_up(A, d) : zshfl_down(A, d);
        const double2 B1 = Fwd ? zshfl_up(B, d) : zshfl_down(B, d);
        if (Fwd ? lane >= d : lane + d < 32) {  // this segment's map after the earlier ones
            B = zfma(A, B1, B);
            A = zmul(A, A1);
        }
    }
    double2 z = Fwd ? zshfl_up(B, 1) : zshfl_down(B, 1);
    if (Fwd ? lane == 0 : lane == 31) z = make_double2(0.0, 0.0);
    for (int i = 0; i < k1 - k0; ++i) {
        const int k = Fwd ? k0 + i : k1 - 1 - i;
        double2 p, q;
        pq(k, p, q);
        z = zfma(q, z, p);
        put(k, z);
    }
}

// Factor the chains of every node update of a level at step size dt (or of
// one solve: nodes = 1, dt = 1, qd.v[0] = alpha).  fac[(i 2 + c) nc + off + k]
// is element k of chain c of wavenumber m (offset off) for node update i;
// one thread per (i, m, c), sequential along the chain.
struct QiDiagC {
    double v[kMaxNodes];
};
__global__ void k_cor_factor(CorFac* __restrict__ fac, const double* __restrict__ cor, int R, int nc, int nodes,
                             QiDiagC qd, double dt, Phys ph, double two_omega) {
    pdl_wait();
    pdl_launch();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nodes * (R + 1) * 2) return;
    const int c = t & 1, m = (t >> 1) % (R + 1), i = (t >> 1) / (R + 1);
    const double alpha = dt * qd.v[i];
    const double sg = two_omega * alpha;
    const int off = moff(R, m), nm = R + 1 - m;
    CorFac* F = fac + ((size_t)i * 2 + c) * nc + off;
    double2 iw_prev = make_double2(0.0, 0.0);
    double sup_prev = 0.0;
    for (int k = 0; k < nm; ++k) {
        const int n = m + k;
        const double L = -n * (n + 1.0) * ph.inv_a2;
        const double cc = 1.0 - alpha * ph.nu * L;
        const double ic = 1.0 / cc;
        const double* cf = cor + 4 * (size_t)(off + k);
        const bool zeta = ((k + c) & 1) == 0;
        const double s = zeta ? sg : -sg;
        const double sub = s * cf[0], sup = s * cf[1];
        double2 w = make_double2(zeta ? cc : cc - alpha * alpha * ph.phibar * L * ic, sg * cf[2]);
        double2 l = make_double2(0.0, 0.0);
        if (k > 0) {
            l = make_double2(sub * iw_prev.x, sub * iw_prev.y);
            w = make_double2(w.x - l.x * sup_prev, w.y - l.y * sup_prev);
        }
        const double2 iw = zrecip(w);
        CorFac e;
        e.l = l;
        e.iw = iw;
        e.u = make_double2(sup * iw.x, sup * iw.y);
        e.ic = ic;
        e.pad = 0.0;
        F[k] = e;
        iw_prev = iw;
        sup_prev = sup;
    }
}

// Solve the two chains of wavenumber m (nm = R + 1 - m unknowns each) from
// the right-hand sides sb[f][k] (f = 0 Phi', 1 zeta, 2 delta; row stride ld)
// into sx[0][k] = zeta_{m+k}, sx[1][k] = delta_{m+k}.  F0 points at element
// (chain 0, k = 0) of this node update's factors, chain 1 is nc further.
// Warps 0 and 1 of the CTA take chains 0 and 1; the caller synchronises.
__device__ __forceinline__ void cor_solve_chains(const double2* sb, double2* sx, int ld, const CorFac* F0, int nc,
                                                 int m, double alpha, const Phys& ph) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp > 1) return;
    const int c = warp;
    const int nm = ld - m;  // ld = R + 1
    const CorFac* F = F0 + (size_t)c * nc;
    // forward substitution y_k = r_k - l_k y_{k-1}; y is kept where x goes
    warp_recurrence<true>(
        nm, lane,
        [&](int k, double2& p, double2& q) {
            const bool zeta = ((k + c) & 1) == 0;
            if (zeta) {
                p = sb[ld + k];
            } else {
                const int n = m + k;
                const double aL = alpha * (-n * (n + 1.0) * ph.inv_a2) * F[k].ic;
                p = make_double2(fma(-aL, sb[k].x, sb[2 * ld + k].x), fma(-aL, sb[k].y, sb[2 * ld + k].y));
            }
            q = zneg(F[k].l);
        },
        [&](int k, double2 y) { sx[(((k + c) & 1) ? ld : 0) + k] = y; });
    // back substitution x_k = iw_k y_k - u_k x_{k+1}
    warp_recurrence<false>(
        nm, lane,
        [&](int k, double2& p, double2& q) {
            p = zmul(F[k].iw, sx[(((k + c) & 1) ? ld : 0) + k]);
            q = zneg(F[k].u);
        },
        [&](int k, double2 x) { sx[(((k + c) & 1) ? ld : 0) + k] = x; });
}

// Phi'_n from the solved delta_n.
__device__ __forceinline__ double2 cor_phi(double2 bp, double2 d, double alpha, const Phys& ph, double ic) {
    return make_double2((bp.x - alpha * ph.phibar * d.x) * ic, (bp.y - alpha * ph.phibar * d.y) * ic);
}

// F_I = L_G + L_F at the coefficients of wavenumber m from the solved values
// in shared memory (sp = Phi', sx = zeta, delta as cor_solve_chains leaves them).
__device__ __forceinline__ void cor_fi_coef(const double2* sx, int ld, const double* cor, int off, int m, int k,
                                            double2 p, const Phys& ph, double two_omega, double2& fp, double2& fz,
                                            double2& fd) {
    const int nm = ld - m, n = m + k;
    const double L = -n * (n + 1.0) * ph.inv_a2;
    const double2 zero = make_double2(0.0, 0.0);
    const double2 zk = sx[k], dk = sx[ld + k];
    implicit_rhs_coef(L, ph, p, zk, dk, fp, fz, fd);
    const double2 zl = k > 0 ? sx[k - 1] : zero, dl = k > 0 ? sx[ld + k - 1] : zero;
    const double2 zu = k + 1 < nm ? sx[k + 1] : zero, du = k + 1 < nm ? sx[ld + k + 1] : zero;
    coriolis_terms(cor + 4 * (size_t)(off + k), zl, zk, zu, dl, dk, du, two_omega, fz, fd);
}

// The node update of an implicit-Coriolis level: right-hand sides b of node
// row.m + 1 (node_rhs, Eq. update_equation_sdcq_discrete_form), the coupled
// solve, and F_I at the new node.  One CTA per (wavenumber m, member).
__global__ void __launch_bounds__(kCorThreads) k_sweep_node_cor(double2* Th, const double2* __restrict__ FIo,
                                                              const double2* __restrict__ FEo, double2* FIn,
                                                              double2* FEn, const double2* __restrict__ tau,
                                                              const CorFac* __restrict__ fac,
                                                              const double* __restrict__ cor, int R, int nc,
                                                              NodeRow row, Phys ph, double two_omega, size_t ms) {
    extern __shared__ double2 cor_sm[];
    pdl_wait();
    pdl_launch();
    const size_t mo = blockIdx.y * ms;
    Th += mo;
    FIo += mo;
    FEo += mo;
    FIn += mo;
    FEn += mo;
    if (tau) tau += mo;
    const int m = blockIdx.x, ld = R + 1, nm = ld - m, off = moff(R, m);
    const size_t node = (size_t)3 * nc;
    double2* sb = cor_sm;           // [3][R+1]
    double2* sx = cor_sm + 3 * ld;  // [2][R+1]
    for (int t = threadIdx.x; t < 3 * nm; t += blockDim.x) {
        const int f = t / nm, k = t - f * nm;
        sb[f * ld + k] = node_rhs(Th, FIo, FEo, FIn, FEn, tau, node, (size_t)f * nc + off + k, row);
    }
    __syncthreads();
    const CorFac* F0 = fac + off;
    cor_solve_chains(sb, sx, ld, F0, nc, m, row.qimm, ph);
    __syncthreads();
    const size_t om = (size_t)(row.m + 1) * node + off;
    for (int k = threadIdx.x; k < nm; k += blockDim.x) {
        const double2 p = cor_phi(sb[k], sx[ld + k], row.qimm, ph, F0[k].ic);
        double2 fp, fz, fd;
        cor_fi_coef(sx, ld, cor, off, m, k, p, ph, two_omega, fp, fz, fd);
        Th[om + k] = p;
        Th[om + nc + k] = sx[k];
        Th[om + 2 * nc + k] = sx[ld + k];
        FIn[om + k] = fp;
        FIn[om + nc + k] = fz;
        FIn[om + 2 * nc + k] = fd;
        if (row.m == 0) {
            for (int f = 0; f < 3; ++f) {
                const size_t o = (size_t)f * nc + off + k;
                FIn[o] = FIo[o];
                FEn[o] = FEo[o];
            }
        }
    }
}

// x = solve(b) for one alpha (factors of one node in fac); x may alias b:
// each CTA reads its wavenumber's coefficients into shared memory before it
// writes them.
__global__ void __launch_bounds__(kCorThreads) k_cor_solve(const double2* b, double2* x,
                                                         const CorFac* __restrict__ fac, int R, int nc, double alpha,
                                                         Phys ph) {
    extern __shared__ double2 cor_sm[];
    pdl_wait();
    pdl_launch();
    const int m = blockIdx.x, ld = R + 1, nm = ld - m, off = moff(R, m);
    double2* sb = cor_sm;
    double2* sx = cor_sm + 3 * ld;
    for (int t = threadIdx.x; t < 3 * nm; t += blockDim.x) {
        const int f = t / nm, k = t - f * nm;
        sb[f * ld + k] = b[(size_t)f * nc + off + k];
    }
    __syncthreads();
    const CorFac* F0 = fac + off;
    cor_solve_chains(sb, sx, ld, F0, nc, m, alpha, ph);
    __syncthreads();
    for (int k = threadIdx.x; k < nm; k += blockDim.x) {
        x[off + k] = cor_phi(sb[k], sx[ld + k], alpha, ph, F0[k].ic);
        x[nc + off + k] = sx[k];
        x[2 * nc + off + k] = sx[ld + k];
    }
}

// F_I = L_G + L_F of `batch` states ms complex values apart; one CTA per
// (wavenumber, state).
__global__ void __launch_bounds__(kCorThreads) k_implicit_rhs_cor(const double2* __restrict__ x,
                                                                double2* __restrict__ F,
                                                                const double* __restrict__ cor, int R, int nc,
                                                                Phys ph, double two_omega, size_t ms) {
    pdl_wait();
    pdl_launch();
    x += blockIdx.y * ms;
    F += blockIdx.y * ms;
    const int m = blockIdx.x, off = moff(R, m), nm = R + 1 - m;
    for (int k = threadIdx.x; k < nm; k += blockDim.x) {
        const int n = m + k;
        const double L = -n * (n + 1.0) * ph.inv_a2;
        const int c = off + k;
        double2 fp, fz, fd;
        implicit_rhs_coef(L, ph, x[c], x[nc + c], x[2 * nc + c], fp, fz, fd);
        coriolis_add(x, cor, nc, R, m, n, off, two_omega, fz, fd);
        F[c] = fp;
        F[nc + c] = fz;
        F[2 * nc + c] = fd;
    }
}

static size_t cor_smem(int R) { return (size_t)5 * (R + 1) * sizeof(double2); }

mlsdc_status cor_smem_limits(int R) {
    mlsdc_status s = raise_smem_limit((const void*)k_sweep_node_cor, cor_smem(R));
    if (s == MLSDC_OK) s = raise_smem_limit((const void*)k_cor_solve, cor_smem(R));
    return s;
}

mlsdc_status cor_factor_launch(sdc_level_t L, double dt, cudaStream_t st) {
    QiDiagC qd{};
    for (int m = 0; m + 1 < L->n; ++m) qd.v[m] = L->QI[(m + 1) * L->n + m + 1];
    const int R = L->plan->R, threads = (L->n - 1) * (R + 1) * 2;
    MLSDC_LAUNCH("k_cor_factor", launch_k(k_cor_factor, dim3((threads + 127) / 128), dim3(128), 0, st, L->d_cfac,
                                          (const double*)L->plan->d_cor, R, L->plan->nc, L->n - 1, qd, dt,
                                          phys_of(L->prm), 2.0 * L->prm.omega));
    L->launches++;
    return MLSDC_OK;
}

mlsdc_status cor_fi_launch(sdc_level_t L, const double2* x, double2* FI, int batch, size_t ms, cudaStream_t st) {
    const int R = L->plan->R;
    MLSDC_LAUNCH("k_implicit_rhs_cor",
                 launch_k(k_implicit_rhs_cor, dim3(R + 1, batch), dim3(kCorThreads), 0, st, x, FI,
                          (const double*)L->plan->d_cor, R, L->plan->nc, phys_of(L->prm), 2.0 * L->prm.omega, ms));
    L->launches++;
    return MLSDC_OK;
}

mlsdc_status cor_node_launch(sdc_level_t L, const NodeRow& row_dt, double2* Th, const double2* FIo,
                             const double2* FEo, double2* FIn, double2* FEn, const double2* tau, cudaStream_t st) {
    const int R = L->plan->R, nc = L->plan->nc;  // shared-memory limit raised at level creation
    MLSDC_LAUNCH("k_sweep_node_cor",
                 launch_k(k_sweep_node_cor, dim3(R + 1, L->members), dim3(kCorThreads), cor_smem(R), st, Th, FIo, FEo,
                          FIn, FEn, tau, (const CorFac*)(L->d_cfac + (size_t)row_dt.m * 2 * nc),
                          (const double*)L->plan->d_cor, R, nc, row_dt, phys_of(L->prm), 2.0 * L->prm.omega, L->ms()));
    L->launches++;
    return MLSDC_OK;
}

}  // namespace mlsdc

using namespace mlsdc;

extern "C" mlsdc_status swe_implicit_rhs_ex(sh_plan_t p, const swe_params* prm, const double* state, double* FI,
                                            int options, void* stream) {
    if (!p || !prm || !state || !FI || (options & ~MLSDC_CORIOLIS_IMPLICIT)) return MLSDC_ERR_INVALID;
    if (!(options & MLSDC_CORIOLIS_IMPLICIT)) return swe_implicit_rhs(p, prm, state, FI, stream);
    k_implicit_rhs_cor<<<dim3(p->R + 1, 1), kCorThreads, 0, (cudaStream_t)stream>>>(
        (const double2*)state, (double2*)FI, p->d_cor, p->R, p->nc, phys_of(*prm), 2.0 * prm->omega, 0);
    MLSDC_LAUNCHED("k_implicit_rhs_cor");
    return MLSDC_OK;
}

extern "C" mlsdc_status swe_implicit_solve_ex(sh_plan_t p, const swe_params* prm, double alpha, const double* b,
                                              double* x, int options, void* stream) {
    if (!p || !prm || !b || !x || !(alpha >= 0.0) || (options & ~MLSDC_CORIOLIS_IMPLICIT)) return MLSDC_ERR_INVALID;
    if (!(options & MLSDC_CORIOLIS_IMPLICIT)) return swe_implicit_solve(p, prm, alpha, b, x, stream);
    cudaStream_t st = (cudaStream_t)stream;
    mlsdc_status s = cor_smem_limits(p->R);
    if (s != MLSDC_OK) return s;
    CorFac* fac = nullptr;
    MLSDC_CUDA(cudaMallocAsync((void**)&fac, (size_t)2 * p->nc * sizeof(CorFac), st));
    QiDiagC qd{};
    qd.v[0] = alpha;
    const int threads = (p->R + 1) * 2;
    k_cor_factor<<<(threads + 127) / 128, 128, 0, st>>>(fac, p->d_cor, p->R, p->nc, 1, qd, 1.0, phys_of(*prm),
                                                       2.0 * prm->omega);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_cor_solve<<<p->R + 1, kCorThreads, cor_smem(p->R), st>>>((const double2*)b, (double2*)x, fac, p->R, p->nc,
                                                                   alpha, phys_of(*prm));
        e = cudaGetLastError();
    }
    cudaFreeAsync(fac, st);
    if (e != cudaSuccess) {
        set_error("k_cor_solve", e);
        return MLSDC_ERR_CUDA;
    }
    return MLSDC_OK;
}
