// IMEX SDC sweeps and two-level MLSDC on the device (Sec. 4.2, Sec. 4.3,
// Algorithm 1), the implicit right-hand side and the per-coefficient implicit
// solve (Sec. 4.4), for one member or a batch of ensemble members advanced in
// lockstep.  All arithmetic here is float64.
//
// Layout: a level with B members holds node arrays [B][M+1][3][nc] (member
// major, so each member's slice is the single-member layout); member b of a
// batched kernel is blockIdx.y and every array advances by its member stride.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "internal.h"
#include "sdc_internal.h"
#include "sdc_kernels.cuh"

namespace mlsdc {


__global__ void k_implicit_rhs(const double2* __restrict__ x, double2* __restrict__ F, const int* __restrict__ ndeg, int nc, Phys ph, size_t ms_x, size_t ms_f) {
    b_implicit_rhs(hw_blk(nullptr), x, F, ndeg, nc, ph, ms_x, ms_f);
}

__global__ void k_implicit_solve(const double2* __restrict__ b, double2* __restrict__ x,
                                 const int* __restrict__ ndeg, int nc, double alpha, Phys ph) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        const double n = ndeg[c];
        const double L = -n * (n + 1.0) * ph.inv_a2;
        double2 p, z, d;
        implicit_solve_coef(L, alpha, ph, b[c], b[nc + c], b[2 * nc + c], p, z, d);
        x[c] = p;
        x[nc + c] = z;
        x[2 * nc + c] = d;
    }
}

// The solve reciprocals of every node update of a sweep at time step dt,
// tab[m][n] = solve_recips(L_n, dt q~I_{m+1,m+1}) for m < M, n <= R.
struct QiDiag {
    double v[kMaxNodes];
};
__global__ void k_solve_coefs(double2* __restrict__ tab, int R, int M, QiDiag qd, double dt, Phys ph) {
    pdl_wait();
    pdl_launch();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < M * (R + 1); t += gridDim.x * blockDim.x) {
        const int m = t / (R + 1), n = t - m * (R + 1);
        tab[t] = solve_recips(-n * (n + 1.0) * ph.inv_a2, dt * qd.v[m], ph);
    }
}

// One SDC node update (Eq. update_equation_sdcq_discrete_form, plus tau on a
// coarse level), the implicit solve, and F_I at the new node.  Node arrays
// are [M+1][3][nc] complex per member (member stride ms); `node` = 3 nc
// complex values.  The m = 0 launch also copies node 0 of the old F arrays
// into the new ones.  Each CTA takes kNodeCoefs coefficients with one thread
// per (field, coefficient) for the weighted sums; the three fields of a
// coefficient meet in shared memory for the coupled solve.
__global__ void __launch_bounds__(3 * kNodeCoefs) k_sweep_node(double2* Th, const double2* __restrict__ FIo, const double2* __restrict__ FEo, double2* FIn, double2* FEn, const double2* __restrict__ tau, const int* __restrict__ ndeg, const double2* __restrict__ recips, int nc, const __grid_constant__ NodeRow row, Phys ph, size_t ms) {
    __shared__ __align__(16) unsigned char smem_nd[kNodeSmem];
    b_sweep_node(hw_blk(smem_nd), Th, FIo, FEo, FIn, FEn, tau, ndeg, recips, nc, row, ph, ms);
}

// The node updates of one sweep with the sweep-constant part gathered once.
// In the update of node r = m + 1 every term that involves only the old
// iterate (the old F arrays), Theta^0 or tau is the same at every node
// update of the sweep (those arrays do not change during it):
//   S_r = Theta^0 + tau_r + sum_{j=0..M} q_rj (FIo_j + FEo_j)
//         - sum_{j=1..r-1} (qE_rj FEo_j + qI_rj FIo_j) - qI_rr FIo_r
// and the update's right-hand side is b_r = S_r + sum_{j=1..r-1} (qE_rj FEn_j
// + qI_rj FIn_j): the terms of Eq. update_equation_sdcq_discrete_form (with
// tau, Eq. modified_update_equation_sdcq_discrete_form) regrouped, the same
// sum up to rounding order.  The m = 0 launch forms S_1..S_M (reading each
// old F array once instead of once per node update), uses S_1 itself and
// keeps S_2..S_M in the level's array S ([members][M-1][3][nc]); the m >= 1
// launches read S_{m+1} and the new values of nodes 1..m only.

template <int MM>
__global__ void __launch_bounds__(3 * kNodeCoefs) k_sweep_node0(double2* Th, const double2* __restrict__ FIo, const double2* __restrict__ FEo, double2* FIn, double2* FEn, const double2* __restrict__ tau, double2* __restrict__ S, const int* __restrict__ ndeg, const double2* __restrict__ recips, int nc, const __grid_constant__ SweepMats sm, Phys ph, size_t ms, size_t ms_s) {
    __shared__ __align__(16) unsigned char smem_nd[kNodeSmem];
    b_sweep_node0<MM>(hw_blk(smem_nd), Th, FIo, FEo, FIn, FEn, tau, S, ndeg, recips, nc, sm, ph, ms, ms_s);
}

// Node update m >= 1 of a sweep whose m = 0 launch (k_sweep_node0) left
// S_{m+1} in S: b = S_{m+1} + sum_{j=1..m} (qE_j FEn_j + qI_j FIn_j), then
// the solve and F_I as k_sweep_node.  `row` is dt_scaled.
__global__ void __launch_bounds__(3 * kNodeCoefs) k_sweep_node_s(double2* Th, double2* FIn, const double2* __restrict__ FEn, const double2* __restrict__ S, const int* __restrict__ ndeg, const double2* __restrict__ recips, int nc, const __grid_constant__ NodeRow row, Phys ph, size_t ms, size_t ms_s) {
    __shared__ __align__(16) unsigned char smem_nd[kNodeSmem];
    b_sweep_node_s(hw_blk(smem_nd), Th, FIn, FEn, S, ndeg, recips, nc, row, ph, ms, ms_s);
}

// dst[k] = src for k = 0..count-1 (node broadcast), src and dst [3 nc] complex
// per member.
__global__ void k_broadcast(const double2* __restrict__ src, double2* __restrict__ dst, int n3, int count, size_t ms_src, size_t ms_dst) {
    b_broadcast(hw_blk(nullptr), src, dst, n3, count, ms_src, ms_dst);
}


// Restriction (Eqs. two_step_restriction, time_restriction, space_restriction):
// Theta_c[i] = D( sum_j Pi^c_f[i][j] Theta_f[j] ) for i in [i0, i1); one
// thread per (coarse node, field, coarse coefficient).
__global__ void k_restrict(const double2* __restrict__ Tf, double2* __restrict__ Tc, const int* __restrict__ c2f, int ncf, int ncc, int nf_nodes, int i0, int i1, const __grid_constant__ TransferMat Pcf, size_t msf, size_t msc) {
    b_restrict(hw_blk(nullptr), Tf, Tc, c2f, ncf, ncc, nf_nodes, i0, i1, Pcf, msf, msc);
}


// tau_c = A_c(R Theta_f) - R A_f(Theta_f) [+ R tau_f], A(Theta) = Theta - dt (Q x I) F
// (Eq. tau_term_level_l+1; tau_f = 0 on the finest level; Eq. collocation_problem), in the
// folded form of FasFwd; one thread per (coarse node i, field, coarse
// coefficient).  The same pass saves the restricted coarse values Theta_c,
// F_I,c, F_E,c (Algorithm 1 step B) into Ts, FIs, FEs for step D.
__global__ void k_fas_tau(const double2* __restrict__ Tf, const double2* __restrict__ FIf, const double2* __restrict__ FEf, const double2* __restrict__ Tc, const double2* __restrict__ FIc, const double2* __restrict__ FEc, double2* __restrict__ tau, double2* __restrict__ Ts, double2* __restrict__ FIs, double2* __restrict__ FEs, const double2* __restrict__ tauf, const int* __restrict__ c2f, int ncf, int ncc, const __grid_constant__ FasFwd A, size_t msf, size_t msc) {
    b_fas_tau(hw_blk(nullptr), Tf, FIf, FEf, Tc, FIc, FEc, tau, Ts, FIs, FEs, tauf, c2f, ncf, ncc, A, msf, msc);
}

// Step D: X_f[m] += P( sum_i Pi^f_c[m][i] (X_c[i] - X_s[i]) ), m = 1..M_f,
// for X = Theta, F_I, F_E (zero-padding leaves the fine-only modes
// unchanged); one thread per (fine node m, field, coarse coefficient), the
// zero weights (fine nodes that are coarse nodes) skipped.
__global__ void k_interp(double2* __restrict__ Tf, double2* __restrict__ FIf, double2* __restrict__ FEf, const double2* __restrict__ Tc, const double2* __restrict__ FIc, const double2* __restrict__ FEc, const double2* __restrict__ Ts, const double2* __restrict__ FIs, const double2* __restrict__ FEs, const int* __restrict__ c2f, int ncf, int ncc, int nfn, int ncn, const __grid_constant__ TransferMat Pfc, size_t msf, size_t msc) {
    b_interp(hw_blk(nullptr), Tf, FIf, FEf, Tc, FIc, FEc, Ts, FIs, FEs, c2f, ncf, ncc, nfn, ncn, Pfc, msf, msc);
}

// X_f += zero-pad(X_c - X_0) at one node per member (X_0 shared by every
// member): the coarse change of a node carried to the fine level without
// interpolation in time; one thread per (field, coarse coefficient).
__global__ void k_pad_add(double2* __restrict__ Xf, const double2* __restrict__ Xc, const double2* __restrict__ X0, const int* __restrict__ c2f, int ncf, int ncc, size_t msf, size_t msc) {
    b_pad_add(hw_blk(nullptr), Xf, Xc, X0, c2f, ncf, ncc, msf, msc);
}

__global__ void k_copy2d(unsigned char* __restrict__ dst, size_t dpitch, const unsigned char* __restrict__ src,
                         size_t spitch, size_t width, int height) {
    b_copy2d(hw_blk(nullptr), dst, dpitch, src, spitch, width, height);
}

// each kernel's recorded arguments are its body's (the persistent kernel
// reads them through the body's parameter list)
MLSDC_SAME_PACK(k_implicit_rhs, b_implicit_rhs);
MLSDC_SAME_PACK(k_sweep_node, b_sweep_node);
MLSDC_SAME_PACK(k_sweep_node0<2>, b_sweep_node0<2>);
MLSDC_SAME_PACK(k_sweep_node_s, b_sweep_node_s);
MLSDC_SAME_PACK(k_broadcast, b_broadcast);
MLSDC_SAME_PACK(k_restrict, b_restrict);
MLSDC_SAME_PACK(k_fas_tau, b_fas_tau);
MLSDC_SAME_PACK(k_interp, b_interp);
MLSDC_SAME_PACK(k_pad_add, b_pad_add);
MLSDC_SAME_PACK(k_copy2d, b_copy2d);

// A device-to-device copy of `height` rows of `width` bytes (cudaMemcpy2DAsync;
// height 1: cudaMemcpyAsync), or under a recorder the copy body of the
// persistent ensemble kernel (16-byte words: every array of a step is complex).
static cudaError_t copy_rows(void* dst, size_t dpitch, const void* src, size_t spitch, size_t width, size_t height,
                             cudaStream_t st) {
    if (Recorder* r = active_recorder()) {
        if (width % 16 || dpitch % 16 || spitch % 16 || (((uintptr_t)dst | (uintptr_t)src) & 15)) {
            r->refused = true;
            return cudaErrorNotSupported;
        }
        const size_t words = width / 16 * height;
        const unsigned blocks = (unsigned)std::max<size_t>(1, std::min<size_t>((words + 255) / 256, 152 * 4));
        record_launch(r, Body::Copy2D, 0, 0, k_copy2d, dim3(blocks), dim3(256), (unsigned char*)dst, dpitch,
                      (const unsigned char*)src, spitch, width, (int)height);
        return cudaSuccess;
    }
    if (height == 1) return cudaMemcpyAsync(dst, src, width, cudaMemcpyDeviceToDevice, st);
    return cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, height, cudaMemcpyDeviceToDevice, st);
}

__global__ void k_finite(const double* __restrict__ x, int64_t n, int* __restrict__ bad) {
    int local = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        local |= !isfinite(x[i]);
    local = __any_sync(0xffffffffu, local);
    if (local && (threadIdx.x & 31) == 0) atomicOr(bad, 1);
}

// ---------------------------------------------------------------------------
// Host-side SDC matrices (Sec. 4.2, Sec. 4.3.3)

static void gauss_nodes(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// n Gauss-Lobatto nodes on [0, 1]: end points and the roots of P'_{n-1}
// (Newton on P'_N with P'' from the Legendre equation), symmetrised.
static std::vector<double> lobatto(int n) {
    const int N = n - 1;
    std::vector<double> x(n);
    x[0] = -1.0;
    x[N] = 1.0;
    const double pi = 3.14159265358979323846;
    for (int i = 1; i < N; ++i) {
        double z = -std::cos(pi * i / N);
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= N; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            const double dP = N * (z * p1 - p0) / (z * z - 1.0);
            const double d2P = (2.0 * z * dP - N * (N + 1.0) * p1) / (1.0 - z * z);
            const double dz = dP / d2P;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
    }
    for (int i = 0; i < n / 2; ++i) {
        const double s = 0.5 * (x[n - 1 - i] - x[i]);
        x[i] = -s;
        x[n - 1 - i] = s;
    }
    if (n % 2 == 1) x[n / 2] = 0.0;
    std::vector<double> t(n);
    for (int i = 0; i < n; ++i) t[i] = 0.5 * (x[i] + 1.0);
    return t;
}

static double lagrange(const std::vector<double>& t, int j, double s) {
    double v = 1.0;
    for (int k = 0; k < (int)t.size(); ++k)
        if (k != j) v *= (s - t[k]) / (t[j] - t[k]);
    return v;
}

}  // namespace mlsdc

using namespace mlsdc;


namespace mlsdc {

// F_E at one node of every member (x and FE point at that node of member 0),
// or, with nodes > 0 on a one-member level, at `nodes` consecutive nodes in
// one launch per stage (the nodes are the batch).
static mlsdc_status eval_FE(sdc_level_t L, const double2* x, double2* FE, cudaStream_t st, int nodes = 0) {
    RhsBatch b;
    b.members = nodes > 0 ? nodes : L->members;
    b.state_ms = b.fe_ms = nodes > 0 ? L->node() : L->ms();
    if (L->plan->precision == MLSDC_FP64)
        return rhs_explicit_f64(L->plan, &L->prm_fe, (const double*)x, (double*)FE, st, &L->launches, -1, b);
    return rhs_explicit_mp(L->plan, &L->prm_fe, (const double*)x, (double*)FE, st, &L->launches, -1, b);
}

static mlsdc_status eval_FI(sdc_level_t L, const double2* x, double2* FI, cudaStream_t st, int nodes = 0) {
    const int nc = L->plan->nc;
    const size_t ms = nodes > 0 ? L->node() : L->ms();
    if (L->options & MLSDC_CORIOLIS_IMPLICIT) return cor_fi_launch(L, x, FI, nodes > 0 ? nodes : L->members, ms, st);
    MLSDC_LAUNCH("k_implicit_rhs", launch_b(Body::ImplicitRhs, 0, 0, k_implicit_rhs, dim3(grid_for(nc), nodes > 0 ? nodes : L->members),
                                            dim3(256), 0, st, x, FI, (const int*)L->plan->d_ndeg, nc,
                                            phys_of(L->prm), ms, ms));
    L->launches++;
    return MLSDC_OK;
}

NodeRow node_row(sdc_level_t L, int m) {
    const int n = L->n;
    NodeRow row;
    std::memset(&row, 0, sizeof(row));
    row.m = m;
    row.M = n - 1;
    for (int j = 0; j < n; ++j) {
        row.qe[j] = L->QE[(m + 1) * n + j];
        row.qi[j] = L->QI[(m + 1) * n + j];
        row.q[j] = L->Q[(m + 1) * n + j];
    }
    row.qimm = L->QI[(m + 1) * n + m + 1];
    return row;
}

static mlsdc_status launch_node(sdc_level_t L, double dt, const NodeRow& row, double2* Th, const double2* FIo,
                                const double2* FEo, double2* FIn, double2* FEn, const double2* tau,
                                cudaStream_t st) {
    if (L->options & MLSDC_CORIOLIS_IMPLICIT)
        return cor_node_launch(L, dt, dt_scaled(row, dt), Th, FIo, FEo, FIn, FEn, tau, st);
    const int nc = L->plan->nc;
    const double2* tab = recips_of(L, dt);
    if (!tab) return invalid_arg("node update: the level's tables for this dt were not prepared");
    const double2* rec = tab + (size_t)row.m * (L->plan->R + 1);
    const dim3 grid((nc + kNodeCoefs - 1) / kNodeCoefs, L->members), block(3 * kNodeCoefs);
    // the sweep-constant terms gathered once per sweep (k_sweep_node0 /
    // k_sweep_node_s); two-node levels have a single update per sweep
    if (L->S) {
        const int M = L->n - 1;
        if (row.m == 0) {
            SweepMats sm;
            std::memset(&sm, 0, sizeof(sm));
            for (int r = 1; r <= M; ++r)
                for (int j = 0; j <= M; ++j) {
                    sm.q[r][j] = dt * L->Q[r * L->n + j];
                    sm.qe[r][j] = dt * L->QE[r * L->n + j];
                    sm.qi[r][j] = dt * L->QI[r * L->n + j];
                }
            const size_t ms_s = (size_t)(M - 1) * L->node();
            cudaError_t e = cudaErrorInvalidValue;
            switch (M) {
#define MLSDC_NODE0(MM)                                                                                          \
    case MM:                                                                                                     \
        e = launch_b((Body)((int)Body::SweepNode0_2 + MM - 2), 0, kNodeSmem, k_sweep_node0<MM>, grid, block, 0, st, Th, FIo, FEo, FIn, FEn, tau, L->S,                   \
                     (const int*)L->plan->d_ndeg, rec, nc, sm, phys_of(L->prm), L->ms(), ms_s);                  \
        break;
                MLSDC_NODE0(2) MLSDC_NODE0(3) MLSDC_NODE0(4) MLSDC_NODE0(5) MLSDC_NODE0(6) MLSDC_NODE0(7)
                MLSDC_NODE0(8)
#undef MLSDC_NODE0
            }
            MLSDC_LAUNCH("k_sweep_node0", e);
        } else {
            MLSDC_LAUNCH("k_sweep_node_s", launch_b(Body::SweepNodeS, 0, kNodeSmem, k_sweep_node_s, grid, block, 0, st, Th, FIn, (const double2*)FEn,
                                                    (const double2*)L->S, (const int*)L->plan->d_ndeg, rec, nc,
                                                    dt_scaled(row, dt), phys_of(L->prm), L->ms(),
                                                    (size_t)(M - 1) * L->node()));
        }
        L->launches++;
        return MLSDC_OK;
    }
    MLSDC_LAUNCH("k_sweep_node",
                 launch_b(Body::SweepNode, 0, kNodeSmem, k_sweep_node, grid, block, 0, st, Th, FIo, FEo, FIn, FEn, tau, (const int*)L->plan->d_ndeg,
                          rec, nc, dt_scaled(row, dt), phys_of(L->prm), L->ms()));
    L->launches++;
    return MLSDC_OK;
}

static mlsdc_status launch_bcast(sdc_level_t L, const double2* src, double2* dst, int n3, int count, size_t ms_src,
                                 size_t ms_dst, cudaStream_t st) {
    MLSDC_LAUNCH("k_broadcast", launch_b(Body::Broadcast, 0, 0, k_broadcast, dim3(grid_for(n3), L->members), dim3(256), 0, st, src, dst, n3,
                                         count, ms_src, ms_dst));
    L->launches++;
    return MLSDC_OK;
}

const double2* recips_of(sdc_level_t L, double dt) {
    for (const auto& e : L->rtab)
        if (e.first == dt) return e.second;
    return nullptr;
}

mlsdc_status solve_recips_for(sdc_level_t L, double dt, cudaStream_t st, const double2** out) {
    if ((*out = recips_of(L, dt))) return MLSDC_OK;
    const int R = L->plan->R;
    double2* buf = nullptr;
    MLSDC_CUDA(cudaMalloc((void**)&buf, (size_t)(L->n - 1) * (R + 1) * sizeof(double2)));
    L->rtab.emplace_back(dt, buf);
    QiDiag qd;
    std::memset(&qd, 0, sizeof(qd));
    for (int m = 0; m + 1 < L->n; ++m) qd.v[m] = L->QI[(m + 1) * L->n + m + 1];
    MLSDC_LAUNCH("k_solve_coefs", launch_k(k_solve_coefs, dim3(grid_for((L->n - 1) * (R + 1))), dim3(256), 0, st,
                                           buf, R, L->n - 1, qd, dt, phys_of(L->prm)));
    L->launches++;
    *out = buf;
    return MLSDC_OK;
}

mlsdc_status prepare_level_tables(sdc_level_t L, double dt, cudaStream_t st) {
    if (L->options & MLSDC_CORIOLIS_IMPLICIT) {
        const CorFac* f = nullptr;
        return cor_factors(L, dt, st, &f);
    }
    const double2* r = nullptr;
    return solve_recips_for(L, dt, st, &r);
}

// The per-dt tables of the level's node updates (solve reciprocals, or with
// implicit Coriolis the factored chains): a launch only the first time a dt
// is seen, nothing afterwards.
static mlsdc_status launch_solve_coefs(sdc_level_t L, double dt, cudaStream_t st) {
    return prepare_level_tables(L, dt, st);
}

// One sweep on explicit buffers ([members][n][3][nc] each).
static mlsdc_status sweep(sdc_level_t L, double dt, double2* Th, const double2* FIo, const double2* FEo,
                          double2* FIn, double2* FEn, const double2* tau, cudaStream_t st) {
    const size_t node = L->node();
    mlsdc_status s0 = launch_solve_coefs(L, dt, st);
    if (s0 != MLSDC_OK) return s0;
    for (int m = 0; m < L->n - 1; ++m) {
        mlsdc_status s = launch_node(L, dt, node_row(L, m), Th, FIo, FEo, FIn, FEn, tau, st);
        if (s != MLSDC_OK) return s;
        s = eval_FE(L, Th + (m + 1) * node, FEn + (m + 1) * node, st);
        if (s != MLSDC_OK) return s;
    }
    return MLSDC_OK;
}

// Initialisation: Theta^n ([members][3][nc]) at every node, F_I and F_E
// evaluated once and spread.
static mlsdc_status spread(sdc_level_t L, const double2* state, cudaStream_t st) {
    const int n3 = (int)L->node();
    mlsdc_status s;
    if ((s = launch_bcast(L, state, L->Th, n3, L->n, (size_t)n3, L->ms(), st)) != MLSDC_OK) return s;
    if ((s = eval_FI(L, L->Th, L->FI[L->cur], st)) != MLSDC_OK) return s;
    if ((s = eval_FE(L, L->Th, L->FE[L->cur], st)) != MLSDC_OK) return s;
    if ((s = launch_bcast(L, L->FI[L->cur], L->FI[L->cur] + n3, n3, L->n - 1, L->ms(), L->ms(), st)) != MLSDC_OK)
        return s;
    return launch_bcast(L, L->FE[L->cur], L->FE[L->cur] + n3, n3, L->n - 1, L->ms(), L->ms(), st);
}

// The last node of every member into state [members][3][nc].
static mlsdc_status copy_last_node(sdc_level_t L, double* state, cudaStream_t st) {
    const size_t w = L->node() * sizeof(double2);
    MLSDC_CUDA(cudaMemcpy2DAsync(state, w, L->Th + (L->n - 1) * L->node(), L->ms() * sizeof(double2), w,
                                 (size_t)L->members, cudaMemcpyDeviceToDevice, st));
    return MLSDC_OK;
}

mlsdc_status implicit_rhs_launch(sh_plan_t p, const swe_params* prm, const double* state, double* FI,
                                 cudaStream_t st) {
    k_implicit_rhs<<<grid_for(p->nc), 256, 0, st>>>((const double2*)state, (double2*)FI, p->d_ndeg, p->nc,
                                                   phys_of(*prm), 0, 0);
    MLSDC_LAUNCHED("k_implicit_rhs");
    return MLSDC_OK;
}

}  // namespace mlsdc



extern "C" mlsdc_status swe_implicit_rhs(sh_plan_t p, const swe_params* prm, const double* state, double* FI,
                                         void* stream) {
    if (!p || !prm || !state || !FI) return MLSDC_ERR_INVALID;
    MLSDC_ALIGNED("swe_implicit_rhs", {"state", state}, {"FI", FI});
    return implicit_rhs_launch(p, prm, state, FI, (cudaStream_t)stream);
}

extern "C" mlsdc_status swe_implicit_solve(sh_plan_t p, const swe_params* prm, double alpha, const double* b,
                                           double* x, void* stream) {
    if (!p || !prm || !b || !x || !(alpha >= 0.0)) return MLSDC_ERR_INVALID;
    MLSDC_ALIGNED("swe_implicit_solve", {"b", b}, {"x", x});
    k_implicit_solve<<<grid_for(p->nc), 256, 0, (cudaStream_t)stream>>>((const double2*)b, (double2*)x, p->d_ndeg,
                                                                       p->nc, alpha, phys_of(*prm));
    MLSDC_LAUNCHED("k_implicit_solve");
    return MLSDC_OK;
}

extern "C" mlsdc_status mlsdc_check_finite(const double* state, int64_t n, int* ok_host, void* stream) {
    if (!state || n < 0 || !ok_host) return MLSDC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    int* d_bad = nullptr;
    MLSDC_CUDA(cudaMallocAsync((void**)&d_bad, sizeof(int), st));
    MLSDC_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int), st));
    k_finite<<<grid_for((int)std::min<int64_t>(n, 1 << 30)), 256, 0, st>>>(state, n, d_bad);
    MLSDC_LAUNCHED("k_finite");
    int bad = 0;
    MLSDC_CUDA(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    MLSDC_CUDA(cudaFreeAsync(d_bad, st));
    MLSDC_CUDA(cudaStreamSynchronize(st));
    *ok_host = bad ? 0 : 1;
    return MLSDC_OK;
}

extern "C" mlsdc_status sdc_level_create_ex(sh_plan_t plan, const swe_params* prm, int n_nodes, int members,
                                            int options, sdc_level_t* out) {
    if (!plan || !prm || !out || n_nodes < 2 || n_nodes > kMaxNodes) return MLSDC_ERR_INVALID;
    if (members < 1 || members > plan->max_members) return MLSDC_ERR_INVALID;
    if (options & ~MLSDC_CORIOLIS_IMPLICIT) return MLSDC_ERR_INVALID;
    sdc_level_t L = new sdc_level_s();
    L->plan = plan;
    L->prm = *prm;
    L->prm_fe = *prm;
    L->options = options;
    if (options & MLSDC_CORIOLIS_IMPLICIT) L->prm_fe.omega = 0.0;  // F_E = N
    L->n = n_nodes;
    L->members = members;
    const int n = n_nodes;
    L->t = lobatto(n);
    L->Q.assign(n * n, 0.0);
    L->QE.assign(n * n, 0.0);
    L->QI.assign(n * n, 0.0);
    std::vector<double> gx, gw;
    gauss_nodes(n, gx, gw);
    for (int m = 0; m < n; ++m)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int q = 0; q < n; ++q) s += gw[q] * lagrange(L->t, j, L->t[m] * (gx[q] + 1.0) / 2.0);
            L->Q[m * n + j] = L->t[m] / 2.0 * s;
        }
    for (int m = 0; m + 1 < n; ++m)
        for (int j = 0; j <= m; ++j) L->QE[(m + 1) * n + j] = L->t[j + 1] - L->t[j];
    // LU trick: (Q[1:,1:])^T = L U (Doolittle), q~I[1:,1:] = U^T
    const int k = n - 1;
    std::vector<double> A(k * k), Lm(k * k, 0.0), U(k * k, 0.0);
    for (int r = 0; r < k; ++r)
        for (int c = 0; c < k; ++c) A[r * k + c] = L->Q[(c + 1) * n + (r + 1)];
    for (int i = 0; i < k; ++i) {
        Lm[i * k + i] = 1.0;
        for (int c = i; c < k; ++c) {
            double s = A[i * k + c];
            for (int q = 0; q < i; ++q) s -= Lm[i * k + q] * U[q * k + c];
            U[i * k + c] = s;
        }
        for (int r = i + 1; r < k; ++r) {
            double s = A[r * k + i];
            for (int q = 0; q < i; ++q) s -= Lm[r * k + q] * U[q * k + i];
            Lm[r * k + i] = s / U[i * k + i];
        }
    }
    for (int r = 0; r < k; ++r)
        for (int c = 0; c < k; ++c) L->QI[(r + 1) * n + (c + 1)] = U[c * k + r];

    const size_t cnt = (size_t)members * L->ms();
    bool ok = cudaMalloc((void**)&L->Th, cnt * sizeof(double2)) == cudaSuccess;
    if (ok && (options & MLSDC_CORIOLIS_IMPLICIT) && cor_smem_limits(plan->R) != MLSDC_OK) {
        sdc_level_destroy(L);
        return MLSDC_ERR_CUDA;
    }
    for (int b = 0; b < 2 && ok; ++b) {
        ok = ok && cudaMalloc((void**)&L->FI[b], cnt * sizeof(double2)) == cudaSuccess;
        ok = ok && cudaMalloc((void**)&L->FE[b], cnt * sizeof(double2)) == cudaSuccess;
    }
    if (ok && n >= 3 && !(options & MLSDC_CORIOLIS_IMPLICIT))
        ok = cudaMalloc((void**)&L->S, (size_t)members * (n - 2) * L->node() * sizeof(double2)) == cudaSuccess;
    if (!ok) {
        set_error("cudaMalloc", cudaGetLastError());
        sdc_level_destroy(L);
        return MLSDC_ERR_ALLOC;
    }
    *out = L;
    return MLSDC_OK;
}

extern "C" mlsdc_status sdc_level_create_batched(sh_plan_t plan, const swe_params* prm, int n_nodes, int members,
                                                 sdc_level_t* out) {
    return sdc_level_create_ex(plan, prm, n_nodes, members, 0, out);
}

extern "C" mlsdc_status sdc_level_create(sh_plan_t plan, const swe_params* prm, int n_nodes, sdc_level_t* out) {
    return sdc_level_create_ex(plan, prm, n_nodes, 1, 0, out);
}

extern "C" mlsdc_status sdc_level_destroy(sdc_level_t L) {
    if (!L) return MLSDC_ERR_INVALID;
    cudaFree(L->Th);
    for (auto& e : L->rtab) cudaFree(e.second);
    cudaFree(L->S);
    for (auto& e : L->cfac) cudaFree(e.second);
    for (int b = 0; b < 2; ++b) {
        cudaFree(L->FI[b]);
        cudaFree(L->FE[b]);
    }
    delete L;
    return MLSDC_OK;
}

extern "C" mlsdc_status sdc_level_matrices(sdc_level_t L, double* t, double* Q, double* QE, double* QI) {
    if (!L) return MLSDC_ERR_INVALID;
    const size_t nn = (size_t)L->n * L->n;
    if (t) std::memcpy(t, L->t.data(), sizeof(double) * L->n);
    if (Q) std::memcpy(Q, L->Q.data(), sizeof(double) * nn);
    if (QE) std::memcpy(QE, L->QE.data(), sizeof(double) * nn);
    if (QI) std::memcpy(QI, L->QI.data(), sizeof(double) * nn);
    return MLSDC_OK;
}

extern "C" mlsdc_status sdc_sweep(sdc_level_t L, double dt, double* Theta, const double* FI_old,
                                  const double* FE_old, double* FI_new, double* FE_new, const double* tau,
                                  void* stream) {
    if (!L || !Theta || !FI_old || !FE_old || !FI_new || !FE_new) return MLSDC_ERR_INVALID;
    if (FI_old == FI_new || FE_old == FE_new) return MLSDC_ERR_INVALID;
    MLSDC_ALIGNED("sdc_sweep", {"Theta", Theta}, {"FI_old", FI_old}, {"FE_old", FE_old}, {"FI_new", FI_new},
                  {"FE_new", FE_new}, {"tau", tau});
    return sweep(L, dt, (double2*)Theta, (const double2*)FI_old, (const double2*)FE_old, (double2*)FI_new,
                 (double2*)FE_new, (const double2*)tau, (cudaStream_t)stream);
}

extern "C" mlsdc_status sdc_step(sdc_level_t L, double* state, double dt, int n_sweeps, void* stream) {
    if (!L || !state || n_sweeps < 0) return MLSDC_ERR_INVALID;
    MLSDC_ALIGNED("sdc_step", {"state", state});
    cudaStream_t st = (cudaStream_t)stream;
    L->launches = 0;
    mlsdc_status s;
    if ((s = spread(L, (const double2*)state, st)) != MLSDC_OK) return s;
    for (int k = 0; k < n_sweeps; ++k) {
        const int c = L->cur;
        if ((s = sweep(L, dt, L->Th, L->FI[c], L->FE[c], L->FI[1 - c], L->FE[1 - c], nullptr, st)) != MLSDC_OK)
            return s;
        L->cur = 1 - c;
    }
    return copy_last_node(L, state, st);
}

extern "C" mlsdc_status mlsdc_profile_node(sdc_level_t L, double dt, int reps, float* ms_out, void* stream) {
    if (!L || !ms_out || reps < 1 || !(dt > 0.0)) return MLSDC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    const int c = L->cur;
    mlsdc_status s = launch_solve_coefs(L, dt, st);
    // a node update reads Theta^0 and the old F arrays and writes node m + 1
    // only, so the repeated launches all do the same work; timed as a graph
    // of `reps` launches, as the step runs them
    for (int m = 0; m < L->n - 1 && s == MLSDC_OK; ++m) {
        const NodeRow row = node_row(L, m);
        s = time_in_graph(st, reps, &ms_out[m], [&](cudaStream_t cs) {
            return launch_node(L, dt, row, L->Th, L->FI[c], L->FE[c], L->FI[1 - c], L->FE[1 - c], nullptr, cs);
        });
    }
    return s;
}

extern "C" mlsdc_status mlsdc_create(sdc_level_t fine, sdc_level_t coarse, mlsdc_t* out) {
    if (!fine || !coarse || !out) return MLSDC_ERR_INVALID;
    if (coarse->plan->R > fine->plan->R || coarse->members != fine->members) return MLSDC_ERR_INVALID;
    if (coarse->options != fine->options) return MLSDC_ERR_INVALID;  // one splitting on both levels
    mlsdc_t ml = new mlsdc_s();
    ml->f = fine;
    ml->c = coarse;
    const int nf = fine->n, ncn = coarse->n;
    std::memset(&ml->Pcf, 0, sizeof(TransferMat));
    std::memset(&ml->Pfc, 0, sizeof(TransferMat));
    for (int i = 0; i < ncn; ++i)
        for (int j = 0; j < nf; ++j) ml->Pcf.a[i * nf + j] = lagrange(fine->t, j, coarse->t[i]);
    for (int m = 0; m < nf; ++m)
        for (int i = 0; i < ncn; ++i) ml->Pfc.a[m * ncn + i] = lagrange(coarse->t, i, fine->t[m]);
    const int Rf = fine->plan->R, Rc = coarse->plan->R;
    std::vector<int> c2f(coarse->plan->nc);
    for (int m = 0; m <= Rc; ++m)
        for (int n = m; n <= Rc; ++n) c2f[moff(Rc, m) + n - m] = moff(Rf, m) + n - m;
    const size_t cnt = (size_t)coarse->members * coarse->ms();
    bool ok = cudaMalloc((void**)&ml->d_c2f, c2f.size() * sizeof(int)) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&ml->Ts, cnt * sizeof(double2)) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&ml->FIs, cnt * sizeof(double2)) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&ml->FEs, cnt * sizeof(double2)) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&ml->tau, cnt * sizeof(double2)) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&ml->cap, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaMemcpy(ml->d_c2f, c2f.data(), c2f.size() * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        set_error("mlsdc_create", cudaGetLastError());
        mlsdc_destroy(ml);
        return MLSDC_ERR_ALLOC;
    }
    *out = ml;
    return MLSDC_OK;
}

extern "C" mlsdc_status mlsdc_destroy(mlsdc_t ml) {
    if (!ml) return MLSDC_ERR_INVALID;
    for (auto& kv : ml->graphs) cudaGraphExecDestroy(kv.second);
    cudaFree(ml->d_c2f);
    cudaFree(ml->Ts);
    cudaFree(ml->FIs);
    cudaFree(ml->FEs);
    cudaFree(ml->tau);
    if (ml->cap) cudaStreamDestroy(ml->cap);
    delete ml;
    return MLSDC_OK;
}

namespace mlsdc {

// The schedule of one MLSDC step (Sec. 4.3.2 initialisation, then Algorithm 1
// steps A-D per iteration) as a list of operations, for L >= 2 levels as the
// V-cycle of mlsdc_step_levels.
size_t build_levels_ops(const std::vector<sdc_level_t>& Lv, const std::vector<mlsdc_t>& pairs, double2* state,
                        double dt, int n_iter, int n_c, std::vector<Op>& ops) {
    const int NL = (int)Lv.size();
    size_t tape = 0;
    ops.clear();
    auto bcast = [&](sdc_level_t L, const double2* src, double2* dst, int count, size_t ms_src) {
        Op o{OpK::Bcast};
        o.L = L;
        o.p[0] = const_cast<double2*>(src);
        o.p[1] = dst;
        o.n3 = (int)L->node();
        o.count = count;
        o.ms_src = ms_src;
        o.ms_dst = L->ms();
        ops.push_back(o);
    };
    auto fi = [&](sdc_level_t L, double2* x, double2* f, int nodes = 0) {
        Op o{OpK::FI};
        o.L = L;
        o.p[0] = x;
        o.p[1] = f;
        o.nodes = nodes;
        ops.push_back(o);
    };
    auto fe = [&](sdc_level_t L, double2* x, double2* f, int nodes = 0) {
        Op o{OpK::FE};
        o.L = L;
        o.p[0] = x;
        o.p[1] = f;
        o.nodes = nodes;
        o.tape_off = tape;
        tape += (size_t)(nodes > 0 ? nodes : L->members) * L->node();
        ops.push_back(o);
    };
    auto sweep_ops = [&](sdc_level_t L, double2* FIo, double2* FEo, double2* FIn, double2* FEn, double2* tau) {
        for (int m = 0; m < L->n - 1; ++m) {
            Op o{OpK::Node};
            o.L = L;
            o.p[0] = L->Th;
            o.p[1] = FIo;
            o.p[2] = FEo;
            o.p[3] = FIn;
            o.p[4] = FEn;
            o.p[5] = tau;
            o.dt = dt;
            o.row = node_row(L, m);
            ops.push_back(o);
            fe(L, L->Th + (m + 1) * L->node(), FEn + (m + 1) * L->node());
        }
    };
    auto restrict_ops = [&](int l, int i0, int i1) {  // level l -> l + 1, coarse nodes [i0, i1)
        Op o{OpK::Restrict};
        o.L = Lv[l + 1];
        o.pair = pairs[l];
        o.p[0] = Lv[l]->Th;
        o.p[1] = Lv[l + 1]->Th;
        o.i0 = i0;
        o.i1 = i1;
        ops.push_back(o);
    };
    std::vector<int> cur(NL);
    for (int l = 0; l < NL; ++l) cur[l] = Lv[l]->cur;
    auto FIc = [&](int l) { return Lv[l]->FI[cur[l]]; };
    auto FEc = [&](int l) { return Lv[l]->FE[cur[l]]; };
    auto sweep_level = [&](int l, double2* tau) {
        sdc_level_t L = Lv[l];
        sweep_ops(L, L->FI[cur[l]], L->FE[cur[l]], L->FI[1 - cur[l]], L->FE[1 - cur[l]], tau);
        cur[l] = 1 - cur[l];
    };
    // the implicit-solve reciprocals (or factored chains) of every level at this dt
    for (sdc_level_t L : Lv) {
        Op o{OpK::SolveCoefs};
        o.L = L;
        o.dt = dt;
        ops.push_back(o);
    }
    // initialisation: fine spread; node 0 of each coarser level = restriction of
    // the level above's node 0, evaluated once
    sdc_level_t F = Lv[0];
    bcast(F, state, F->Th, F->n, F->node());
    fi(F, F->Th, FIc(0));
    fe(F, F->Th, FEc(0));
    bcast(F, FIc(0), FIc(0) + F->node(), F->n - 1, F->ms());
    bcast(F, FEc(0), FEc(0) + F->node(), F->n - 1, F->ms());
    for (int l = 1; l < NL; ++l) {
        restrict_ops(l - 1, 0, 1);
        fi(Lv[l], Lv[l]->Th, FIc(l));
        fe(Lv[l], Lv[l]->Th, FEc(l));
    }
    for (int it = 0; it < n_iter; ++it) {
        // A) fine sweep
        sweep_level(0, nullptr);
        for (int l = 0; l + 1 < NL; ++l) {
            const int c = l + 1;
            sdc_level_t C = Lv[c];
            const size_t nodec = C->node();
            const int ncn = C->n;
            // B) restrict nodes 1..Mc, evaluate, save.  The evaluations at the
            // coarse nodes are independent: with one member and a coarse plan
            // sized for them, all Mc nodes go in one launch per stage.
            restrict_ops(l, 1, ncn);
            if (C->members == 1 && ncn > 2 && C->plan->max_members >= ncn - 1) {
                fi(C, C->Th + nodec, FIc(c) + nodec, ncn - 1);
                fe(C, C->Th + nodec, FEc(c) + nodec, ncn - 1);
            } else {
                for (int i = 1; i < ncn; ++i) {
                    fi(C, C->Th + i * nodec, FIc(c) + i * nodec);
                    fe(C, C->Th + i * nodec, FEc(c) + i * nodec);
                }
            }
            // C) FAS correction (its pass also saves the restricted values of
            // step B), coarse sweeps
            mlsdc_t P = pairs[l];
            Op fa{OpK::Fas};
            fa.L = C;
            fa.pair = P;
            fa.tauf = l > 0 ? pairs[l - 1]->tau : nullptr;
            double2* fas[10] = {Lv[l]->Th, FIc(l), FEc(l), C->Th, FIc(c), FEc(c), P->tau, P->Ts, P->FIs, P->FEs};
            std::copy(fas, fas + 10, fa.p);
            fa.dt = dt;
            ops.push_back(fa);
            for (int k = 0; k < n_c; ++k) sweep_level(c, P->tau);
        }
        // D) back up: interpolate each level's corrections to the level above,
        // one sweep on every intermediate level
        for (int l = NL - 2; l >= 0; --l) {
            const int c = l + 1;
            mlsdc_t P = pairs[l];
            Op ip{OpK::Interp};
            ip.L = Lv[c];
            ip.pair = P;
            double2* ipp[9] = {Lv[l]->Th, FIc(l), FEc(l), Lv[c]->Th, FIc(c), FEc(c), P->Ts, P->FIs, P->FEs};
            std::copy(ipp, ipp + 9, ip.p);
            ops.push_back(ip);
            if (l > 0) sweep_level(l, pairs[l - 1]->tau);
        }
    }
    Op last{OpK::CopyLast};
    last.L = F;
    last.p[0] = F->Th + (F->n - 1) * F->node();
    last.p[1] = state;
    ops.push_back(last);
    for (int l = 0; l < NL; ++l) Lv[l]->cur = cur[l];
    return tape;
}

size_t build_mlsdc_ops(mlsdc_t ml, double2* state, double dt, int n_iter, int n_c, std::vector<Op>& ops) {
    return build_levels_ops({ml->f, ml->c}, {ml}, state, dt, n_iter, n_c, ops);
}

mlsdc_status run_ops(mlsdc_t ml, const std::vector<Op>& ops, cudaStream_t st, int64_t* launches, double2* tape) {
    // every level the operations touch (launch accounting)
    std::vector<sdc_level_t> lv;
    for (const Op& o : ops)
        if (o.L && std::find(lv.begin(), lv.end(), o.L) == lv.end()) lv.push_back(o.L);
    for (sdc_level_t L : lv) L->launches = 0;
    int64_t own = 0;
    mlsdc_status s = MLSDC_OK;
    Recorder* rec = active_recorder();
    for (size_t oi = 0; oi < ops.size(); ++oi) {
        const Op& o = ops[oi];
        if (rec) rec->begin_op((int)oi);
        // the level pair of a transfer operation (the two-level object by default)
        const mlsdc_s* P = o.pair ? o.pair : ml;
        sdc_level_t F = P->f, C = P->c;
        const int ncf = F->plan->nc, ncc = C->plan->nc;
        const int nfn = F->n, ncn = C->n;
        const size_t msf = F->ms(), msc = C->ms();
        auto gt = [&](int threads) { return dim3(grid_for(threads), F->members); };
        switch (o.k) {
            case OpK::Bcast:
                s = launch_bcast(o.L, o.p[0], o.p[1], o.n3, o.count, o.ms_src, o.ms_dst, st);
                break;
            case OpK::FI:
                s = eval_FI(o.L, o.p[0], o.p[1], st, o.nodes);
                break;
            case OpK::FE:
                if (tape && o.nodes > 0) {
                    MLSDC_CUDA(cudaMemcpyAsync(tape + o.tape_off, o.p[0], (size_t)o.nodes * o.L->node() * sizeof(double2),
                                               cudaMemcpyDeviceToDevice, st));
                } else if (tape) {
                    const size_t w = o.L->node() * sizeof(double2);
                    MLSDC_CUDA(cudaMemcpy2DAsync(tape + o.tape_off, w, o.p[0], o.L->ms() * sizeof(double2), w,
                                                 (size_t)o.L->members, cudaMemcpyDeviceToDevice, st));
                }
                s = eval_FE(o.L, o.p[0], o.p[1], st, o.nodes);
                break;
            case OpK::Node:
                s = launch_node(o.L, o.dt, o.row, o.p[0], o.p[1], o.p[2], o.p[3], o.p[4], o.p[5], st);
                break;
            case OpK::Restrict:
                MLSDC_LAUNCH("k_restrict",
                             launch_b(Body::Restrict, 0, 0, k_restrict, gt((o.i1 - o.i0) * 3 * ncc), dim3(256), 0, st, o.p[0], o.p[1],
                                      (const int*)P->d_c2f, ncf, ncc, nfn, o.i0, o.i1, P->Pcf, msf, msc));
                own++;
                break;
            case OpK::Copy:
                MLSDC_CUDA(copy_rows(o.p[1], o.bytes, o.p[0], o.bytes, o.bytes, 1, st));
                break;
            case OpK::Fas: {
                FasFwd fw;
                std::memset(&fw, 0, sizeof(fw));
                fw.nfn = nfn;
                fw.ncn = ncn;
                for (int i = 0; i < ncn; ++i) {
                    for (int j = 0; j < nfn; ++j) {
                        double pq = 0.0;
                        for (int l = 0; l < nfn; ++l) pq += P->Pcf.a[i * nfn + l] * F->Q[l * nfn + j];
                        fw.Pcf[i * nfn + j] = P->Pcf.a[i * nfn + j];
                        fw.dPQf[i * nfn + j] = o.dt * pq;
                    }
                    for (int l = 0; l < ncn; ++l) fw.dQc[i * ncn + l] = o.dt * C->Q[i * ncn + l];
                }
                MLSDC_LAUNCH("k_fas_tau", launch_b(Body::FasTau, 0, 0, k_fas_tau, gt(ncn * 3 * ncc), dim3(256), 0, st, o.p[0], o.p[1],
                                                   o.p[2], o.p[3], o.p[4], o.p[5], o.p[6], o.p[7], o.p[8], o.p[9],
                                                   (const double2*)o.tauf, (const int*)P->d_c2f, ncf, ncc, fw, msf,
                                                   msc));
                own++;
                break;
            }
            case OpK::Interp:
                MLSDC_LAUNCH("k_interp",
                             launch_b(Body::Interp, 0, 0, k_interp, gt((nfn - 1) * 3 * ncc), dim3(256), 0, st, o.p[0], o.p[1], o.p[2],
                                      o.p[3], o.p[4], o.p[5], o.p[6], o.p[7], o.p[8], (const int*)P->d_c2f, ncf, ncc,
                                      nfn, ncn, P->Pfc, msf, msc));
                own++;
                break;
            case OpK::SolveCoefs:
                s = launch_solve_coefs(o.L, o.dt, st);
                break;
            case OpK::CopyLast: {
                const size_t w = o.L->node() * sizeof(double2);
                MLSDC_CUDA(copy_rows(o.p[1], w, o.p[0], o.L->ms() * sizeof(double2), w, (size_t)o.L->members, st));
                break;
            }
            case OpK::Copy2D:
                MLSDC_CUDA(copy_rows(o.p[1], o.ms_dst * sizeof(double2), o.p[0], o.ms_src * sizeof(double2), o.bytes,
                                     (size_t)o.count, st));
                break;
            case OpK::PadAdd:
                MLSDC_LAUNCH("k_pad_add", launch_b(Body::PadAdd, 0, 0, k_pad_add, dim3(grid_for(3 * ncc), o.count), dim3(256), 0, st,
                                                   o.p[0], (const double2*)o.p[1], (const double2*)o.p[2],
                                                   (const int*)P->d_c2f, ncf, ncc, msf, msc));
                own++;
                break;
        }
        if (s != MLSDC_OK) return s;
    }
    if (launches) {
        *launches = own;
        for (sdc_level_t L : lv) *launches += L->launches;
    }
    return MLSDC_OK;
}

// Work a step at dt needs done once, outside any graph capture: the
// factored Coriolis chains of implicit-Coriolis levels.
mlsdc_status prepare_levels(mlsdc_t ml, double dt, cudaStream_t st) {
    for (sdc_level_t L : {ml->f, ml->c}) {
        mlsdc_status s = prepare_level_tables(L, dt, st);
        if (s != MLSDC_OK) return s;
    }
    return MLSDC_OK;
}

static mlsdc_status mlsdc_enqueue(mlsdc_t ml, double* state, double dt, int n_iter, int n_c, cudaStream_t st) {
    std::vector<Op> ops;
    build_mlsdc_ops(ml, (double2*)state, dt, n_iter, n_c, ops);
    return run_ops(ml, ops, st, &ml->launches, nullptr);
}

// Capture `enqueue(stream)` once into an executable graph.
template <class Enqueue>
static mlsdc_status capture(cudaStream_t cap, cudaGraphExec_t* out, Enqueue enqueue) {
    MLSDC_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    mlsdc_status s = enqueue(cap);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &g);
    if (s != MLSDC_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) {
        set_error("cudaStreamEndCapture", e);
        return MLSDC_ERR_CUDA;
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        set_error("cudaGraphInstantiate", e);
        return MLSDC_ERR_CUDA;
    }
    return MLSDC_OK;
}

}  // namespace mlsdc

extern "C" mlsdc_status mlsdc_step(mlsdc_t ml, double* state, double dt, int n_iter, int n_coarse_sweeps,
                                   int use_graph, void* stream) {
    if (!ml || !state || n_iter < 0 || n_coarse_sweeps < 0) return MLSDC_ERR_INVALID;
    MLSDC_ALIGNED("mlsdc_step", {"state", state});
    cudaStream_t st = (cudaStream_t)stream;
    mlsdc_status sp = prepare_levels(ml, dt, st);
    if (sp != MLSDC_OK) return sp;
    if (!use_graph) return mlsdc_enqueue(ml, state, dt, n_iter, n_coarse_sweeps, st);
    auto key = std::make_tuple(state, dt, n_iter, n_coarse_sweeps);
    auto it = ml->graphs.find(key);
    if (it == ml->graphs.end()) {
        // The F ping-pong parity must be the same at every replay: it is,
        // because each step flips each level's buffer a fixed number of times;
        // reset both to 0 so capture and replays agree.
        ml->f->cur = 0;
        ml->c->cur = 0;
        cudaGraphExec_t ex = nullptr;
        mlsdc_status s = capture(ml->cap, &ex, [&](cudaStream_t cs) {
            return mlsdc_enqueue(ml, state, dt, n_iter, n_coarse_sweeps, cs);
        });
        if (s != MLSDC_OK) return s;
        it = ml->graphs.emplace(key, ex).first;
        ml->f->cur = 0;
        ml->c->cur = 0;
    }
    MLSDC_CUDA(cudaGraphLaunch(it->second, st));
    return MLSDC_OK;
}

// ------------------------------------------------------- three or more levels
struct mlsdc_levels_s {
    std::vector<sdc_level_t> levels;
    std::vector<mlsdc_t> pairs;  // pairs[l] joins levels l and l + 1 (owned)
    cudaStream_t cap = nullptr;
    std::map<std::tuple<double*, double, int, int>, cudaGraphExec_t> graphs;
    int64_t launches = 0;
};

extern "C" mlsdc_status mlsdc_levels_destroy(mlsdc_levels_t h) {
    if (!h) return MLSDC_ERR_INVALID;
    for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
    for (mlsdc_t p : h->pairs) mlsdc_destroy(p);
    if (h->cap) cudaStreamDestroy(h->cap);
    delete h;
    return MLSDC_OK;
}

extern "C" mlsdc_status mlsdc_levels_create(const sdc_level_t* levels, int n_levels, mlsdc_levels_t* out) {
    if (!levels || !out || n_levels < 2 || n_levels > 8) return MLSDC_ERR_INVALID;
    for (int l = 0; l < n_levels; ++l) {
        if (!levels[l]) return MLSDC_ERR_INVALID;
        for (int k = 0; k < l; ++k)
            if (levels[k] == levels[l]) return MLSDC_ERR_INVALID;  // each level's node arrays are its own
    }
    mlsdc_levels_t h = new mlsdc_levels_s();
    h->levels.assign(levels, levels + n_levels);
    for (int l = 0; l + 1 < n_levels; ++l) {
        mlsdc_t p = nullptr;
        mlsdc_status s = mlsdc_create(levels[l], levels[l + 1], &p);
        if (s != MLSDC_OK) {
            mlsdc_levels_destroy(h);
            return s;
        }
        h->pairs.push_back(p);
    }
    if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) {
        set_error("mlsdc_levels_create", cudaGetLastError());
        mlsdc_levels_destroy(h);
        return MLSDC_ERR_CUDA;
    }
    *out = h;
    return MLSDC_OK;
}

namespace mlsdc {
static mlsdc_status levels_enqueue(mlsdc_levels_t h, double* state, double dt, int n_iter, int n_c, cudaStream_t st) {
    std::vector<Op> ops;
    build_levels_ops(h->levels, h->pairs, (double2*)state, dt, n_iter, n_c, ops);
    return run_ops(h->pairs[0], ops, st, &h->launches, nullptr);
}
}  // namespace mlsdc

extern "C" mlsdc_status mlsdc_levels_step(mlsdc_levels_t h, double* state, double dt, int n_iter, int n_coarse_sweeps,
                                          int use_graph, void* stream) {
    if (!h || !state || n_iter < 0 || n_coarse_sweeps < 0) return MLSDC_ERR_INVALID;
    MLSDC_ALIGNED("mlsdc_levels_step", {"state", state});
    cudaStream_t st = (cudaStream_t)stream;
    for (mlsdc_t p : h->pairs) {
        mlsdc_status sp = prepare_levels(p, dt, st);
        if (sp != MLSDC_OK) return sp;
    }
    if (!use_graph) return levels_enqueue(h, state, dt, n_iter, n_coarse_sweeps, st);
    auto key = std::make_tuple(state, dt, n_iter, n_coarse_sweeps);
    auto it = h->graphs.find(key);
    if (it == h->graphs.end()) {
        for (sdc_level_t L : h->levels) L->cur = 0;  // the same buffer parity at capture and every replay
        cudaGraphExec_t ex = nullptr;
        mlsdc_status s = capture(h->cap, &ex, [&](cudaStream_t cs) {
            return levels_enqueue(h, state, dt, n_iter, n_coarse_sweeps, cs);
        });
        if (s != MLSDC_OK) return s;
        it = h->graphs.emplace(key, ex).first;
        for (sdc_level_t L : h->levels) L->cur = 0;
    }
    MLSDC_CUDA(cudaGraphLaunch(it->second, st));
    return MLSDC_OK;
}

extern "C" mlsdc_status mlsdc_levels_launch_count(mlsdc_levels_t h, int64_t* launches) {
    if (!h || !launches) return MLSDC_ERR_INVALID;
    *launches = h->launches;
    return MLSDC_OK;
}

extern "C" mlsdc_status mlsdc_launch_count(mlsdc_t ml, int64_t* launches) {
    if (!ml || !launches) return MLSDC_ERR_INVALID;
    *launches = ml->launches;
    return MLSDC_OK;
}

// ------------------------------------------------------------------ ensemble
extern "C" mlsdc_status mlsdc_ensemble_create(const mlsdc_t* groups, int ngroups, mlsdc_ensemble_t* out) {
    if (!groups || ngroups < 1 || ngroups > 64 || !out) return MLSDC_ERR_INVALID;
    for (int g = 0; g < ngroups; ++g)
        if (!groups[g]) return MLSDC_ERR_INVALID;
    mlsdc_ensemble_t e = new mlsdc_ensemble_s();
    e->groups.assign(groups, groups + ngroups);
    bool ok = cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int g = 0; g < ngroups && ok; ++g) {
        cudaStream_t s;
        cudaEvent_t ev;
        ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
        if (ok) {
            e->streams.push_back(s);
            e->done.push_back(ev);
        }
    }
    if (!ok) {
        set_error("mlsdc_ensemble_create", cudaGetLastError());
        mlsdc_ensemble_destroy(e);
        return MLSDC_ERR_CUDA;
    }
    *out = e;
    return MLSDC_OK;
}

extern "C" mlsdc_status mlsdc_ensemble_destroy(mlsdc_ensemble_t e) {
    if (!e) return MLSDC_ERR_INVALID;
    for (auto& kv : e->graphs) cudaGraphExecDestroy(kv.second);
    for (auto s : e->streams) cudaStreamDestroy(s);
    for (auto ev : e->done) cudaEventDestroy(ev);
    if (e->fork) cudaEventDestroy(e->fork);
    if (e->cap) cudaStreamDestroy(e->cap);
    persistent_free(e);
    delete e;
    return MLSDC_OK;
}

namespace mlsdc {

// Fork: every group's step runs on its own stream after `st`; join: `st`
// waits for all of them.  Inside a capture this becomes one graph with one
// branch per group.
static mlsdc_status ensemble_enqueue(mlsdc_ensemble_t e, const std::vector<double*>& states, double dt, int n_iter,
                                     int n_c, cudaStream_t st) {
    MLSDC_CUDA(cudaEventRecord(e->fork, st));
    e->launches = 0;
    for (size_t g = 0; g < e->groups.size(); ++g) {
        MLSDC_CUDA(cudaStreamWaitEvent(e->streams[g], e->fork, 0));
        mlsdc_status s = mlsdc_enqueue(e->groups[g], states[g], dt, n_iter, n_c, e->streams[g]);
        if (s != MLSDC_OK) return s;
        e->launches += e->groups[g]->launches;
        MLSDC_CUDA(cudaEventRecord(e->done[g], e->streams[g]));
        MLSDC_CUDA(cudaStreamWaitEvent(st, e->done[g], 0));
    }
    return MLSDC_OK;
}

}  // namespace mlsdc

extern "C" mlsdc_status mlsdc_ensemble_step(mlsdc_ensemble_t e, double* const* states, double dt, int n_iter,
                                            int n_coarse_sweeps, int use_graph, void* stream) {
    if (!e || !states || n_iter < 0 || n_coarse_sweeps < 0) return MLSDC_ERR_INVALID;
    std::vector<double*> sv(states, states + e->groups.size());
    for (double* p : sv) {
        if (!p) return MLSDC_ERR_INVALID;
        MLSDC_ALIGNED("mlsdc_ensemble_step", {"states[i]", p});
    }
    cudaStream_t st = (cudaStream_t)stream;
    for (mlsdc_t ml : e->groups) {
        mlsdc_status sp = prepare_levels(ml, dt, st);
        if (sp != MLSDC_OK) return sp;
    }
    if (!use_graph) return ensemble_enqueue(e, sv, dt, n_iter, n_coarse_sweeps, st);
    auto key = std::make_tuple(sv, dt, n_iter, n_coarse_sweeps);
    auto it = e->graphs.find(key);
    if (it == e->graphs.end()) {
        for (mlsdc_t ml : e->groups) ml->f->cur = ml->c->cur = 0;
        cudaGraphExec_t ex = nullptr;
        mlsdc_status s = capture(e->cap, &ex, [&](cudaStream_t cs) {
            return ensemble_enqueue(e, sv, dt, n_iter, n_coarse_sweeps, cs);
        });
        if (s != MLSDC_OK) return s;
        it = e->graphs.emplace(key, ex).first;
        for (mlsdc_t ml : e->groups) ml->f->cur = ml->c->cur = 0;
    }
    MLSDC_CUDA(cudaGraphLaunch(it->second, st));
    return MLSDC_OK;
}

extern "C" mlsdc_status mlsdc_ensemble_launch_count(mlsdc_ensemble_t e, int64_t* launches) {
    if (!e || !launches) return MLSDC_ERR_INVALID;
    *launches = e->launches;
    return MLSDC_OK;
}
