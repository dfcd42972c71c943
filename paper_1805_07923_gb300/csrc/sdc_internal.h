// Internal declarations of the time-stepping part of the library (SDC levels,
// two-level MLSDC, the step's operation list), shared by the forward step
// (sdc.cu) and its adjoint (adjoint.cu).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <tuple>
#include <vector>

#include "internal.h"
#include "node_update.cuh"

namespace mlsdc {

constexpr int kNodeCoefs = 64;  // coefficients per CTA of the node update (3 x 64 threads)

// Time interpolation matrix between two node sets (Sec. 4.3.3).
struct TransferMat {
    double a[kMaxNodes * kMaxNodes];
};

struct FasArgs {
    double Qf[kMaxNodes * kMaxNodes];
    double Qc[kMaxNodes * kMaxNodes];
    double Pcf[kMaxNodes * kMaxNodes];
    int nfn, ncn;
};

// The forward FAS pass's matrices for one step size dt, formed on the host:
// Pcf, dt Q_c and dt Pcf Q_f, so that
//   tau_i = Theta_c,i - sum_j Pcf_ij Theta_f,j - sum_l (dt Q_c)_il F_c,l + sum_j (dt Pcf Q_f)_ij F_f,j
// (F = F_I + F_E; the same value as A_c(R Theta_f) - R A_f(Theta_f) with the
// fine sums folded through Pcf).
struct FasFwd {
    double Pcf[kMaxNodes * kMaxNodes];   // [ncn][nfn]
    double dQc[kMaxNodes * kMaxNodes];   // [ncn][ncn]
    double dPQf[kMaxNodes * kMaxNodes];  // [ncn][nfn]
    int nfn, ncn;
};

// One operation of an MLSDC step.  A step is a fixed, straight-line list of
// these (built on the host from the schedule of Algorithm 1), run in order
// by the forward step and walked backwards by the adjoint.  Every operation
// except FE is linear in its operands with constant coefficients.
enum class OpK : int {
    Bcast,     // p[1][k] = p[0] for k < count                (node broadcast, spread)
    FI,        // p[1] = F_I(p[0])                              (one node, every member)
    FE,        // p[1] = F_E(p[0])
    Node,      // k_sweep_node: node m+1 update, solve, F_I     (p: Th FIo FEo FIn FEn tau)
    Restrict,  // coarse p[1][i] = D(sum_j Pcf[i][j] p[0][j]), i in [i0, i1)
    Copy,      // p[1] = p[0], `bytes` bytes
    Fas,       // tau (p[6]) from fine (p[0..2]) and coarse (p[3..5]) nodes; saves p[3..5] to p[7..9]
    Interp,    // fine p[0..2] += P(Pfc (coarse p[3..5] - saved p[6..8]))
    CopyLast,  // p[1] (the state) = last fine node p[0], every member
    SolveCoefs,  // the level's implicit-solve reciprocals at dt (no state operands)
    Copy2D,    // `count` rows of `bytes` bytes, p[0] -> p[1], row pitches ms_src / ms_dst (complex values)
    PadAdd,    // fine p[0] += zero-pad(coarse p[1] - p[2]) at one node, `count` members from p[0], p[1]
               // (member strides of the pair's levels; p[2] the same for every member)
};

struct Op {
    OpK k;
    sdc_level_t L = nullptr;         // the level the operation runs on
    double2* p[10] = {};             // operands, by kind (above)
    int n3 = 0, count = 0;           // Bcast
    size_t ms_src = 0, ms_dst = 0;   // Bcast member strides
    int i0 = 0, i1 = 0;              // Restrict
    size_t bytes = 0;                // Copy
    double dt = 0.0;                 // Node, Fas
    NodeRow row{};                   // Node
    size_t tape_off = 0;             // FE: offset of its linearisation point in a step's tape (complex)
    int nodes = 0;                   // FI / FE: > 0 = that many consecutive nodes of a one-member level
                                     // in one launch (the nodes as the batch); 0 = one node of every member
    mlsdc_t pair = nullptr;          // Restrict / Fas / Interp: the level pair (fine, coarse) they join
    double2* tauf = nullptr;         // Fas: the finer level's own tau (null on the finest pair)
};

inline Phys phys_of(const swe_params& p) { return Phys{1.0 / (p.a * p.a), p.phibar, p.nu}; }

// Row m + 1 of level L's SDC matrices (not yet scaled by dt).
NodeRow node_row(sdc_level_t L, int m);

// One element of a factored Coriolis chain (coriolis_implicit.cu): the
// Thomas elimination's multiplier l, the pivot's reciprocal iw and the
// scaled super-diagonal u = c iw; ic = 1/c_n with c_n = 1 - alpha nu L_n, and
// aLc = alpha L_n / c_n (the factor of b_Phi in a delta row's right-hand side).
struct CorFac {
    double2 l, iw, u;
    double ic, aLc;
};

// The implicit-Coriolis splitting (coriolis_implicit.cu).  Levels created
// with MLSDC_CORIOLIS_IMPLICIT evaluate F_E with Omega = 0 and F_I with the
// Coriolis terms; their node updates solve the coupled system per m.
// The factored chains depend only on the level and dt: a level keeps one
// set per step size it has seen (cor_factors computes a new one on `st`;
// the step entry points call it before any graph capture, so a captured step
// only reads them).
mlsdc_status cor_smem_limits(int R);  // once per level, outside any graph capture
mlsdc_status cor_factors(sdc_level_t L, double dt, cudaStream_t st, const CorFac** out);
mlsdc_status cor_factor_launch(sdc_level_t L, double dt, cudaStream_t st);
mlsdc_status cor_fi_launch(sdc_level_t L, const double2* x, double2* FI, int batch, size_t ms, cudaStream_t st);
mlsdc_status cor_node_launch(sdc_level_t L, double dt, const NodeRow& row_dt, double2* Th, const double2* FIo,
                             const double2* FEo, double2* FIn, double2* FEn, const double2* tau, cudaStream_t st);

// The solve reciprocals of level L's node updates at step size dt ([n-1][R+1],
// node-major): looked up, or computed on `st` the first time dt is seen
// (allocates; call outside stream capture).  recips_of returns the table of
// an already prepared dt, or nullptr.
mlsdc_status solve_recips_for(sdc_level_t L, double dt, cudaStream_t st, const double2** out);
const double2* recips_of(sdc_level_t L, double dt);
// Every per-dt table a step of level L at dt reads (solve reciprocals, or the
// factored Coriolis chains): prepared outside graph capture.
mlsdc_status prepare_level_tables(sdc_level_t L, double dt, cudaStream_t st);


inline int grid_for(int n) {
    int b = (n + 255) / 256;
    return b < 1 ? 1 : (b > 152 * 8 ? 152 * 8 : b);
}

}  // namespace mlsdc

struct sdc_level_s {
    sh_plan_t plan;
    swe_params prm;
    swe_params prm_fe;  // the parameters F_E is evaluated with (Omega = 0 with implicit Coriolis)
    int options = 0;    // MLSDC_CORIOLIS_IMPLICIT
    int n;        // nodes
    int members;  // ensemble members advanced together
    std::vector<double> t, Q, QE, QI;
    double2* Th = nullptr;  // [members][n][3][nc]
    double2* FI[2] = {nullptr, nullptr};
    double2* FE[2] = {nullptr, nullptr};
    // per step size dt, the solve reciprocals of the node updates [n-1][R+1]
    // (k_solve_coefs): computed the first time a dt is seen, before any graph
    // capture, and kept, so a step's graph only reads them
    std::vector<std::pair<double, double2*>> rtab;
    // the sweep-constant parts S_2..S_M of the node updates' right-hand sides,
    // [members][n-2][3][nc] (k_sweep_node0 writes them, k_sweep_node_s reads;
    // null for two nodes and for the implicit-Coriolis splitting)
    double2* S = nullptr;
    // implicit Coriolis only: per step size dt, the factored chains [n-1][2][nc]
    std::vector<std::pair<double, mlsdc::CorFac*>> cfac;
    int cur = 0;
    int64_t launches = 0;
    size_t node() const { return (size_t)3 * plan->nc; }
    size_t ms() const { return (size_t)n * node(); }  // member stride of node arrays
};

struct mlsdc_s {
    sdc_level_t f, c;
    mlsdc::TransferMat Pcf, Pfc;
    int* d_c2f = nullptr;
    double2 *Ts = nullptr, *FIs = nullptr, *FEs = nullptr, *tau = nullptr;
    cudaStream_t cap = nullptr;
    std::map<std::tuple<double*, double, int, int>, cudaGraphExec_t> graphs;
    int64_t launches = 0;
};

struct mlsdc_ensemble_s {
    std::vector<mlsdc_t> groups;
    std::vector<cudaStream_t> streams;  // one per group (fork-join branches)
    std::vector<cudaEvent_t> done;      // one per group
    cudaEvent_t fork = nullptr;
    cudaStream_t cap = nullptr;
    std::map<std::tuple<std::vector<double*>, double, int, int>, cudaGraphExec_t> graphs;
    int64_t launches = 0;
    void* persist = nullptr;  // the persistent-kernel form of the step (persistent.cu)
};

namespace mlsdc {

// Release the persistent-kernel state of an ensemble (persistent.cu).
void persistent_free(mlsdc_ensemble_t e);

// Work a step at dt needs done once, outside any graph capture (the
// per-dt tables of both levels).
mlsdc_status prepare_levels(mlsdc_t ml, double dt, cudaStream_t st);

// The operations of one MLSDC step on `state` (Algorithm 1, n_iter
// iterations of one fine and n_c coarse sweeps), starting from the levels'
// current buffer parities, which it advances as the step will.  Returns the
// number of complex values one step's F_E linearisation points take.
size_t build_mlsdc_ops(mlsdc_t ml, double2* state, double dt, int n_iter, int n_c, std::vector<Op>& ops);

// The same for L >= 2 levels (levels[0] finest), pairs[l] joining levels l
// and l + 1: the V-cycle of mlsdc_step_levels (down: restrict, evaluate,
// FAS with the restricted finer tau, n_c sweeps; up: interpolate, one sweep
// on each intermediate level).  With two levels the list is build_mlsdc_ops's.
size_t build_levels_ops(const std::vector<sdc_level_t>& levels, const std::vector<mlsdc_t>& pairs, double2* state,
                        double dt, int n_iter, int n_c, std::vector<Op>& ops);

// Launch the operations in order on `st`.  With `tape`, each FE operation
// first copies its input to tape + tape_off.
mlsdc_status run_ops(mlsdc_t ml, const std::vector<Op>& ops, cudaStream_t st, int64_t* launches, double2* tape);

}  // namespace mlsdc
