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

constexpr int kCorThreads = 256;      // standalone solve and F_I: per wavenumber, warps 0 and 1 solve the chains
constexpr int kCorNodeThreads = 128;  // node update: per (wavenumber, chain), warp 0 solves

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

// The same recurrence over all warps of the CTA (blockDim.x threads, a
// multiple of 32): thread t takes positions [t s, t s + s) of the recurrence
// order (k ascending for Fwd, descending otherwise), s = ceil(n / blockDim.x);
// each warp scans its lanes' maps, warp totals meet in shared memory
// (wsum[2 * warps]), and every thread then runs its segment from its carry.
// pq(k, p, q) is called once per k (the first pass keeps p in pbuf[k]);
// called by every thread of the CTA (it synchronises).
template <bool Fwd, class PQ, class Put>
__device__ __forceinline__ void block_recurrence(int n, PQ pq, Put put, double2* pbuf, double2* wsum) {
    const int T = blockDim.x, t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = T >> 5;
    const int s = (n + T - 1) / T;
    const int j0 = min(n, t * s), j1 = min(n, j0 + s);
    double2 A = make_double2(1.0, 0.0), B = make_double2(0.0, 0.0);
    for (int j = j0; j < j1; ++j) {
        const int k = Fwd ? j : n - 1 - j;
        double2 p, q;
        pq(k, p, q);
        pbuf[k] = p;
        B = zfma(q, B, p);
        A = zmul(q, A);
    }
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const double2 A1 = zshfl_up(A, d), B1 = zshfl_up(B, d);
        if (lane >= d) {
            B = zfma(A, B1, B);
            A = zmul(A, A1);
        }
    }
    if (lane == 31) {
        wsum[warp] = A;
        wsum[nw + warp] = B;
    }
    __syncthreads();
    double2 z = make_double2(0.0, 0.0);  // the value before this warp's first position
    for (int w = 0; w < warp; ++w) z = zfma(wsum[w], z, wsum[nw + w]);
    double2 Ae = zshfl_up(A, 1), Be = zshfl_up(B, 1);
    if (lane > 0) z = zfma(Ae, z, Be);
    for (int j = j0; j < j1; ++j) {
        const int k = Fwd ? j : n - 1 - j;
        double2 p, q;
        pq(k, p, q);
        z = zfma(q, z, pbuf[k]);
        put(k, z);
    }
    __syncthreads();
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
        e.aLc = alpha * L * ic;
        F[k] = e;
        iw_prev = iw;
        sup_prev = sup;
    }
}

// Solve the two chains of wavenumber m (nm = R + 1 - m unknowns each) from
// the right-hand sides sb[f][k] (f = 0 Phi', 1 zeta, 2 delta; row stride ld)
// into sx[0][k] = zeta_{m+k}, sx[1][k] = delta_{m+k}.  sf holds this node
// update's factors of chain 0 (sf[k]) and chain 1 (sf[ld + k]) in shared
// memory.  Warps 0 and 1 of the CTA take chains 0 and 1; the caller
// synchronises.
__device__ __forceinline__ void cor_solve_chains(const double2* sb, double2* sx, int ld, const CorFac* sf, int m,
                                                 double alpha, const Phys& ph) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp > 1) return;
    const int c = warp;
    const int nm = ld - m;  // ld = R + 1
    const CorFac* F = sf + c * ld;
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

// Copy this wavenumber's factors of both chains (global fac: chain 0 at
// F0[k], chain 1 at F0[nc + k]) into shared memory sf[c ld + k], 16 bytes per
// thread and step.
__device__ __forceinline__ void cor_stage_factors(CorFac* sf, const CorFac* __restrict__ F0, int nc, int ld, int nm) {
    constexpr int kV = sizeof(CorFac) / sizeof(double2);
    for (int t = threadIdx.x; t < 2 * nm * kV; t += blockDim.x) {
        const int c = t / (nm * kV), r = t - c * nm * kV;
        reinterpret_cast<double2*>(sf + c * ld)[r] = reinterpret_cast<const double2*>(F0 + (size_t)c * nc)[r];
    }
}

// Phi'_n from the solved delta_n.
__device__ __forceinline__ double2 cor_phi(double2 bp, double2 d, double alpha, const Phys& ph, double ic) {
    return make_double2((bp.x - alpha * ph.phibar * d.x) * ic, (bp.y - alpha * ph.phibar * d.y) * ic);
}

// The node update of an implicit-Coriolis level: right-hand sides b of node
// row.m + 1 (node_rhs, Eq. update_equation_sdcq_discrete_form), the coupled
// solve, and F_I at the new node.  One CTA per (wavenumber m, chain c,
// member): chain c holds zeta_{m+k} for k + c even and delta_{m+k} for k + c
// odd, and every value the outputs of its elements need is in the chain
// (F_I of zeta_n uses delta_{n-1}, delta_{n+1}; F_I of delta_n and Phi'_n use
// zeta_{n-1}, zeta_{n+1} and Phi'_n, which comes from delta_n), so the two
// chains of a wavenumber run on different SMs without exchanging anything.
__global__ void __launch_bounds__(kCorNodeThreads) k_sweep_node_cor(double2* Th, const double2* __restrict__ FIo,
                                                                  const double2* __restrict__ FEo, double2* FIn,
                                                                  double2* FEn, const double2* __restrict__ tau,
                                                                  const CorFac* __restrict__ fac,
                                                                  const double* __restrict__ cor, int R, int nc,
                                                                  NodeRow row, Phys ph, double two_omega, size_t ms) {
    extern __shared__ double2 cor_sm[];
    pdl_wait();
    pdl_launch();
    const size_t mo = blockIdx.z * ms;
    Th += mo;
    FIo += mo;
    FEo += mo;
    FIn += mo;
    FEn += mo;
    if (tau) tau += mo;
    const int m = blockIdx.x, c = blockIdx.y, ld = R + 1, nm = ld - m, off = moff(R, m);
    const size_t node = (size_t)3 * nc;
    const double alpha = row.qimm;
    double2* sr = cor_sm;                                     // [R+1] b_zeta or b_delta of element k
    double2* sp = cor_sm + ld;                                // [R+1] b_Phi at the delta elements
    double2* sx = cor_sm + 2 * ld;                            // [R+1] the chain's solution
    double2* pb = cor_sm + 3 * ld;                            // [R+1] the recurrences' p_k
    double2* ws = cor_sm + 4 * ld;                            // [2 warps] warp totals
    CorFac* sf = reinterpret_cast<CorFac*>(cor_sm + 4 * ld + 2 * (kCorNodeThreads / 32));  // [R+1] factors
    {
        constexpr int kV = sizeof(CorFac) / sizeof(double2);
        const double2* src = reinterpret_cast<const double2*>(fac + (size_t)c * nc + off);
        for (int t = threadIdx.x; t < nm * kV; t += blockDim.x) reinterpret_cast<double2*>(sf)[t] = src[t];
    }
    for (int t = threadIdx.x; t < 2 * nm; t += blockDim.x) {
        const int k = t >> 1, second = t & 1;
        const bool zeta = ((k + c) & 1) == 0;
        if (zeta && second) continue;
        const int f = zeta ? 1 : (second ? 0 : 2);
        const double2 b = node_rhs(Th, FIo, FEo, FIn, FEn, tau, node, (size_t)f * nc + off + k, row);
        (second ? sp : sr)[k] = b;
    }
    __syncthreads();
    // forward substitution y_k = r_k - l_k y_{k-1} (the delta rows with Phi'
    // eliminated: r = b_delta - alpha L_n b_Phi / c_n), then back substitution
    // x_k = iw_k y_k - u_k x_{k+1}; y and x are kept in sx
    block_recurrence<true>(
        nm,
        [&](int k, double2& p, double2& q) {
            if (((k + c) & 1) == 0) {
                p = sr[k];
            } else {
                const double aL = sf[k].aLc;
                p = make_double2(fma(-aL, sp[k].x, sr[k].x), fma(-aL, sp[k].y, sr[k].y));
            }
            q = zneg(sf[k].l);
        },
        [&](int k, double2 y) { sx[k] = y; }, pb, ws);
    block_recurrence<false>(
        nm,
        [&](int k, double2& p, double2& q) {
            p = zmul(sf[k].iw, sx[k]);
            q = zneg(sf[k].u);
        },
        [&](int k, double2 x) { sx[k] = x; }, pb, ws);
    const size_t om = (size_t)(row.m + 1) * node + off;
    const double2 zero = make_double2(0.0, 0.0);
    for (int k = threadIdx.x; k < nm; k += blockDim.x) {
        const int n = m + k;
        const double L = -n * (n + 1.0) * ph.inv_a2;
        const double nl = ph.nu * L;
        const double* cf = cor + 4 * (size_t)(off + k);
        const double2 v = sx[k];
        const double2 lo = k > 0 ? sx[k - 1] : zero, hi = k + 1 < nm ? sx[k + 1] : zero;
        if (((k + c) & 1) == 0) {  // zeta_n: nu L zeta + L_F (delta_{n-1}, zeta_n, delta_{n+1})
            double2 fz = make_double2(nl * v.x, nl * v.y);
            coriolis_zeta_row(cf, lo, v, hi, two_omega, fz);
            Th[om + nc + k] = v;
            FIn[om + nc + k] = fz;
        } else {  // delta_n and Phi'_n: L_G, and L_F (zeta_{n-1}, delta_n, zeta_{n+1})
            const double2 p = cor_phi(sp[k], v, alpha, ph, sf[k].ic);
            const double2 fp = make_double2(-ph.phibar * v.x + nl * p.x, -ph.phibar * v.y + nl * p.y);
            double2 fd = make_double2(-L * p.x + nl * v.x, -L * p.y + nl * v.y);
            coriolis_delta_row(cf, lo, v, hi, two_omega, fd);
            Th[om + k] = p;
            Th[om + 2 * nc + k] = v;
            FIn[om + k] = fp;
            FIn[om + 2 * nc + k] = fd;
        }
        if (row.m == 0 && c == 0) {
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
    CorFac* sf = reinterpret_cast<CorFac*>(cor_sm + 5 * ld);
    cor_stage_factors(sf, fac + off, nc, ld, nm);
    for (int t = threadIdx.x; t < 3 * nm; t += blockDim.x) {
        const int f = t / nm, k = t - f * nm;
        sb[f * ld + k] = b[(size_t)f * nc + off + k];
    }
    __syncthreads();
    cor_solve_chains(sb, sx, ld, sf, m, alpha, ph);
    __syncthreads();
    for (int k = threadIdx.x; k < nm; k += blockDim.x) {
        x[off + k] = cor_phi(sb[k], sx[ld + k], alpha, ph, sf[k].ic);
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

// standalone solve: right-hand sides [3][R+1], solution [2][R+1], factors [2][R+1]
static size_t cor_smem(int R) { return (size_t)5 * (R + 1) * sizeof(double2) + (size_t)2 * (R + 1) * sizeof(CorFac); }
// node update, one chain: r, b_Phi, solution, p [R+1] each, warp totals, factors [R+1]
static size_t cor_node_smem(int R) {
    return (size_t)(4 * (R + 1) + 2 * (kCorNodeThreads / 32)) * sizeof(double2) + (size_t)(R + 1) * sizeof(CorFac);
}

mlsdc_status cor_smem_limits(int R) {
    mlsdc_status s = raise_smem_limit((const void*)k_sweep_node_cor, cor_node_smem(R));
    if (s == MLSDC_OK) s = raise_smem_limit((const void*)k_cor_solve, cor_smem(R));
    return s;
}

mlsdc_status cor_factors(sdc_level_t L, double dt, cudaStream_t st, const CorFac** out) {
    for (const auto& e : L->cfac)
        if (e.first == dt) {
            *out = e.second;
            return MLSDC_OK;
        }
    CorFac* buf = nullptr;
    MLSDC_CUDA(cudaMalloc((void**)&buf, (size_t)(L->n - 1) * 2 * L->plan->nc * sizeof(CorFac)));
    L->cfac.emplace_back(dt, buf);
    QiDiagC qd{};
    for (int m = 0; m + 1 < L->n; ++m) qd.v[m] = L->QI[(m + 1) * L->n + m + 1];
    const int R = L->plan->R, threads = (L->n - 1) * (R + 1) * 2;
    MLSDC_LAUNCH("k_cor_factor", launch_k(k_cor_factor, dim3((threads + 127) / 128), dim3(128), 0, st, buf,
                                          (const double*)L->plan->d_cor, R, L->plan->nc, L->n - 1, qd, dt,
                                          phys_of(L->prm), 2.0 * L->prm.omega));
    L->launches++;
    *out = buf;
    return MLSDC_OK;
}

mlsdc_status cor_factor_launch(sdc_level_t L, double dt, cudaStream_t st) {
    const CorFac* f = nullptr;
    return cor_factors(L, dt, st, &f);
}

mlsdc_status cor_fi_launch(sdc_level_t L, const double2* x, double2* FI, int batch, size_t ms, cudaStream_t st) {
    const int R = L->plan->R;
    MLSDC_LAUNCH("k_implicit_rhs_cor",
                 launch_k(k_implicit_rhs_cor, dim3(R + 1, batch), dim3(kCorThreads), 0, st, x, FI,
                          (const double*)L->plan->d_cor, R, L->plan->nc, phys_of(L->prm), 2.0 * L->prm.omega, ms));
    L->launches++;
    return MLSDC_OK;
}

mlsdc_status cor_node_launch(sdc_level_t L, double dt, const NodeRow& row_dt, double2* Th, const double2* FIo,
                             const double2* FEo, double2* FIn, double2* FEn, const double2* tau, cudaStream_t st) {
    const int R = L->plan->R, nc = L->plan->nc;  // shared-memory limit raised at level creation
    const CorFac* fac = nullptr;
    mlsdc_status s = cor_factors(L, dt, st, &fac);
    if (s != MLSDC_OK) return s;
    MLSDC_LAUNCH("k_sweep_node_cor",
                 launch_k(k_sweep_node_cor, dim3(R + 1, 2, L->members), dim3(kCorNodeThreads), cor_node_smem(R), st,
                          Th, FIo, FEo, FIn, FEn, tau, fac + (size_t)row_dt.m * 2 * nc, (const double*)L->plan->d_cor,
                          R, nc, row_dt, phys_of(L->prm), 2.0 * L->prm.omega, L->ms()));
    L->launches++;
    return MLSDC_OK;
}

}  // namespace mlsdc

using namespace mlsdc;

extern "C" mlsdc_status swe_implicit_rhs_ex(sh_plan_t p, const swe_params* prm, const double* state, double* FI,
                                            int options, void* stream) {
    if (!p || !prm || !state || !FI || (options & ~MLSDC_CORIOLIS_IMPLICIT)) return MLSDC_ERR_INVALID;
    MLSDC_ALIGNED("swe_implicit_rhs_ex", {"state", state}, {"FI", FI});
    if (!(options & MLSDC_CORIOLIS_IMPLICIT)) return swe_implicit_rhs(p, prm, state, FI, stream);
    k_implicit_rhs_cor<<<dim3(p->R + 1, 1), kCorThreads, 0, (cudaStream_t)stream>>>(
        (const double2*)state, (double2*)FI, p->d_cor, p->R, p->nc, phys_of(*prm), 2.0 * prm->omega, 0);
    MLSDC_LAUNCHED("k_implicit_rhs_cor");
    return MLSDC_OK;
}

extern "C" mlsdc_status swe_implicit_solve_ex(sh_plan_t p, const swe_params* prm, double alpha, const double* b,
                                              double* x, int options, void* stream) {
    if (!p || !prm || !b || !x || !(alpha >= 0.0) || (options & ~MLSDC_CORIOLIS_IMPLICIT)) return MLSDC_ERR_INVALID;
    MLSDC_ALIGNED("swe_implicit_solve_ex", {"b", b}, {"x", x});
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
