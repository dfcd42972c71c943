// Two-level PFASST on one GPU: P time slices advanced together, each slice
// one member of the batched fine and coarse levels.
//
// The paper names PFASST (the parallel full approximation scheme in space and
// time) as the time-parallel extension of its two-level MLSDC (Sec. 1 and the
// conclusions) without printing it; this follows the published two-level
// iteration, built on the library's Algorithm 1 steps A-D.  Slice p covers
// [t0 + p dt, t0 + (p+1) dt].  What runs in parallel across slices runs as
// one member-batched launch per kernel: the fine sweeps, the restriction and
// coarse evaluations, the FAS correction and the interpolation.  The coarse
// sweeps run slice after slice, each starting from the coarse end value the
// slice before it produced in the same iteration (the pipeline's serial
// part); a slice's fine initial value is the fine end value of the slice
// before it from the previous iteration.
//
// Predictor: every slice's fine nodes start as u0; the coarse level runs
// serially over the slices (slice 0 from R u0, slice p from slice p-1's
// coarse end value, each spread and swept n_pred times); slices p >= 1 then
// start from v_p = u0 + pad(coarse initial value - R u0), spread with F
// evaluated.  Slice 0 is then exactly Algorithm 1's MLSDC step.
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "internal.h"
#include "sdc_internal.h"

struct pfasst_s {
    mlsdc_t pair = nullptr;                 // the two batched levels (owned pair object)
    int P = 0;                              // time slices = members of both levels
    std::vector<sdc_level_s*> cview;        // the coarse level, one slice each (views into its arrays)
    double2* Ru0 = nullptr;                 // [3][nc_c] R u0
    cudaStream_t cap = nullptr;
    std::map<std::tuple<const double*, double*, double, int, int, int>, cudaGraphExec_t> graphs;
    int64_t launches = 0;
};

namespace mlsdc {
namespace {

// A one-member view of member p of a batched level: the same plan, tables
// and matrices; the node arrays (and the sweep-constant array S) start at
// member p.  Views own nothing.
void make_view(const sdc_level_s* L, int p, sdc_level_s* V) {
    *V = *L;
    V->members = 1;
    const size_t ms = L->ms();
    V->Th = L->Th + p * ms;
    for (int b = 0; b < 2; ++b) {
        V->FI[b] = L->FI[b] + p * ms;
        V->FE[b] = L->FE[b] + p * ms;
    }
    if (L->S) V->S = L->S + (size_t)p * (L->n - 2) * L->node();
}

struct Builder {
    pfasst_s* pf;
    double dt;
    std::vector<Op>& ops;

    void bcast(sdc_level_t L, double2* src, double2* dst, int count, size_t ms_src) {
        Op o{OpK::Bcast};
        o.L = L;
        o.p[0] = src;
        o.p[1] = dst;
        o.n3 = (int)L->node();
        o.count = count;
        o.ms_src = ms_src;
        o.ms_dst = L->ms();
        ops.push_back(o);
    }
    void eval(OpK k, sdc_level_t L, double2* x, double2* F, int nodes = 0) {
        Op o{k};
        o.L = L;
        o.p[0] = x;
        o.p[1] = F;
        o.nodes = nodes;
        ops.push_back(o);
    }
    void copy(double2* src, double2* dst, size_t n) {
        Op o{OpK::Copy};
        o.p[0] = src;
        o.p[1] = dst;
        o.bytes = n * sizeof(double2);
        ops.push_back(o);
    }
    void copy2d(double2* src, double2* dst, size_t n, int rows, size_t pitch) {
        Op o{OpK::Copy2D};
        o.p[0] = src;
        o.p[1] = dst;
        o.bytes = n * sizeof(double2);
        o.count = rows;
        o.ms_src = o.ms_dst = pitch;
        ops.push_back(o);
    }
    // node 0 -> nodes 1..M with F_I, F_E evaluated at node 0 and spread
    void spread_node0(sdc_level_t L, double2* FI, double2* FE) {
        bcast(L, L->Th, L->Th + L->node(), L->n - 1, L->ms());
        eval(OpK::FI, L, L->Th, FI);
        eval(OpK::FE, L, L->Th, FE);
        bcast(L, FI, FI + L->node(), L->n - 1, L->ms());
        bcast(L, FE, FE + L->node(), L->n - 1, L->ms());
    }
    // one sweep on L (all its members) from the F arrays of parity c
    void sweep(sdc_level_t L, int c, const double2* tau) {
        Op sc{OpK::SolveCoefs};
        sc.L = L;
        sc.dt = dt;
        ops.push_back(sc);
        for (int m = 0; m + 1 < L->n; ++m) {
            Op o{OpK::Node};
            o.L = L;
            o.p[0] = L->Th;
            o.p[1] = L->FI[c];
            o.p[2] = L->FE[c];
            o.p[3] = L->FI[1 - c];
            o.p[4] = L->FE[1 - c];
            o.p[5] = (double2*)tau;
            o.dt = dt;
            o.row = node_row(L, m);
            ops.push_back(o);
            eval(OpK::FE, L, L->Th + (m + 1) * L->node(), L->FE[1 - c] + (m + 1) * L->node());
        }
    }
    void restrict_nodes(int i0, int i1) {
        Op o{OpK::Restrict};
        o.L = pf->pair->c;
        o.pair = pf->pair;
        o.p[0] = pf->pair->f->Th;
        o.p[1] = pf->pair->c->Th;
        o.i0 = i0;
        o.i1 = i1;
        ops.push_back(o);
    }
};

void build_pfasst_ops(pfasst_s* pf, const double* u0, double* ends, double dt, int n_iter, int n_c, int n_pred,
                      std::vector<Op>& ops) {
    Builder b{pf, dt, ops};
    mlsdc_t pr = pf->pair;
    sdc_level_t F = pr->f, C = pr->c;
    const int P = pf->P;
    const size_t nodeF = F->node(), nodeC = C->node(), msF = F->ms(), msC = C->ms();
    int fc = 0, cc = 0;  // buffer parities (every slice sweeps equally often, so one per level)
    // ---- predictor
    b.bcast(F, (double2*)u0, F->Th, F->n, 0);
    b.restrict_nodes(0, 1);
    b.copy(C->Th, pf->Ru0, nodeC);
    for (int p = 0; p < P; ++p) {
        sdc_level_t V = pf->cview[p];
        if (p > 0) b.copy(pf->cview[p - 1]->Th + (C->n - 1) * nodeC, V->Th, nodeC);
        int c = cc;
        b.spread_node0(V, V->FI[c], V->FE[c]);
        for (int s = 0; s < n_pred; ++s) {
            b.sweep(V, c, nullptr);
            c = 1 - c;
        }
    }
    if (n_pred & 1) cc = 1 - cc;
    if (P > 1) {
        Op pa{OpK::PadAdd};
        pa.L = C;
        pa.pair = pr;
        pa.p[0] = F->Th + msF;
        pa.p[1] = C->Th + msC;
        pa.p[2] = pf->Ru0;
        pa.count = P - 1;
        ops.push_back(pa);
    }
    b.spread_node0(F, F->FI[fc], F->FE[fc]);
    // ---- iterations
    const bool batched_coarse = C->plan->max_members >= P * C->n;
    for (int k = 0; k < n_iter; ++k) {
        // A) fine initial values from the previous iteration, then one fine sweep of every slice
        if (k > 0 && P > 1) {
            b.copy2d(F->Th + (F->n - 1) * nodeF, F->Th + msF, nodeF, P - 1, msF);
            b.eval(OpK::FI, F, F->Th, F->FI[fc]);
            b.eval(OpK::FE, F, F->Th, F->FE[fc]);
        }
        b.sweep(F, fc, nullptr);
        fc = 1 - fc;
        // B) restrict nodes 0..M_c, evaluate at every coarse node of every slice
        b.restrict_nodes(0, C->n);
        if (batched_coarse) {
            b.eval(OpK::FI, C, C->Th, C->FI[cc], P * C->n);
            b.eval(OpK::FE, C, C->Th, C->FE[cc], P * C->n);
        } else {
            for (int i = 0; i < C->n; ++i) {
                b.eval(OpK::FI, C, C->Th + i * nodeC, C->FI[cc] + i * nodeC);
                b.eval(OpK::FE, C, C->Th + i * nodeC, C->FE[cc] + i * nodeC);
            }
        }
        // FAS correction of every slice (its pass also saves the restricted values)
        Op fa{OpK::Fas};
        fa.L = C;
        fa.pair = pr;
        double2* fas[10] = {F->Th, F->FI[fc], F->FE[fc], C->Th, C->FI[cc], C->FE[cc], pr->tau, pr->Ts, pr->FIs, pr->FEs};
        std::copy(fas, fas + 10, fa.p);
        fa.dt = dt;
        ops.push_back(fa);
        // C) the coarse pipeline: slice p starts from slice p-1's coarse end value
        for (int p = 0; p < P; ++p) {
            sdc_level_t V = pf->cview[p];
            int c = cc;
            if (p > 0) {
                b.copy(pf->cview[p - 1]->Th + (C->n - 1) * nodeC, V->Th, nodeC);
                b.eval(OpK::FI, V, V->Th, V->FI[c]);
                b.eval(OpK::FE, V, V->Th, V->FE[c]);
            }
            for (int s = 0; s < n_c; ++s) {
                b.sweep(V, c, pr->tau + p * msC);
                c = 1 - c;
            }
        }
        if (n_c & 1) cc = 1 - cc;
        // D) interpolate every slice's coarse corrections to its fine nodes 1..M_f
        Op ip{OpK::Interp};
        ip.L = C;
        ip.pair = pr;
        double2* ipp[9] = {F->Th, F->FI[fc], F->FE[fc], C->Th, C->FI[cc], C->FE[cc], pr->Ts, pr->FIs, pr->FEs};
        std::copy(ipp, ipp + 9, ip.p);
        ops.push_back(ip);
    }
    Op last{OpK::CopyLast};
    last.L = F;
    last.p[0] = F->Th + (F->n - 1) * nodeF;
    last.p[1] = (double2*)ends;
    ops.push_back(last);
}

mlsdc_status pfasst_enqueue(pfasst_s* pf, const double* u0, double* ends, double dt, int n_iter, int n_c, int n_pred,
                            cudaStream_t st) {
    std::vector<Op> ops;
    build_pfasst_ops(pf, u0, ends, dt, n_iter, n_c, n_pred, ops);
    return run_ops(pf->pair, ops, st, &pf->launches, nullptr);
}

}  // namespace
}  // namespace mlsdc

using namespace mlsdc;

extern "C" mlsdc_status pfasst_create(sdc_level_t fine, sdc_level_t coarse, pfasst_t* out) {
    if (!fine || !coarse || !out) return invalid_arg("pfasst_create: null argument");
    if (fine->members != coarse->members)
        return invalid_arg("pfasst_create: both levels need one member per time slice");
    if (fine->options || coarse->options)
        return invalid_arg("pfasst_create: only the paper's splitting (Coriolis in F_E) is supported");
    pfasst_s* pf = new pfasst_s();
    pf->P = fine->members;
    mlsdc_status s = mlsdc_create(fine, coarse, &pf->pair);
    if (s != MLSDC_OK) {
        delete pf;
        return s;
    }
    for (int p = 0; p < pf->P; ++p) {
        sdc_level_s* v = new sdc_level_s();
        make_view(coarse, p, v);
        pf->cview.push_back(v);
    }
    bool ok = cudaMalloc((void**)&pf->Ru0, coarse->node() * sizeof(double2)) == cudaSuccess &&
              cudaStreamCreateWithFlags(&pf->cap, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) {
        set_error("pfasst_create", cudaGetLastError());
        pfasst_destroy(pf);
        return MLSDC_ERR_ALLOC;
    }
    *out = pf;
    return MLSDC_OK;
}

extern "C" mlsdc_status pfasst_destroy(pfasst_t pf) {
    if (!pf) return MLSDC_ERR_INVALID;
    for (auto& kv : pf->graphs) cudaGraphExecDestroy(kv.second);
    for (sdc_level_s* v : pf->cview) {
        v->rtab.clear();  // views share their level's tables
        v->cfac.clear();
        delete v;
    }
    if (pf->pair) mlsdc_destroy(pf->pair);
    cudaFree(pf->Ru0);
    if (pf->cap) cudaStreamDestroy(pf->cap);
    delete pf;
    return MLSDC_OK;
}

extern "C" mlsdc_status pfasst_step(pfasst_t pf, const double* u0, double* ends, double dt, int n_iter,
                                    int n_coarse_sweeps, int n_predictor_sweeps, int use_graph, void* stream) {
    if (!pf || !u0 || !ends) return invalid_arg("pfasst_step: null argument");
    if (n_iter < 0 || n_coarse_sweeps < 0 || !(dt > 0.0))
        return invalid_arg("pfasst_step: n_iter and n_coarse_sweeps must be >= 0 and dt > 0");
    MLSDC_ALIGNED("pfasst_step", {"u0", u0}, {"ends", ends});
    const int n_pred = n_predictor_sweeps < 0 ? n_coarse_sweeps : n_predictor_sweeps;
    cudaStream_t st = (cudaStream_t)stream;
    sdc_level_t F = pf->pair->f, C = pf->pair->c;
    for (sdc_level_t L : {F, C}) {
        mlsdc_status s = prepare_level_tables(L, dt, st);
        if (s != MLSDC_OK) return s;
    }
    for (sdc_level_s* v : pf->cview) v->rtab = C->rtab;  // the coarse level's per-dt tables
    F->cur = C->cur = 0;
    if (!use_graph) return pfasst_enqueue(pf, u0, ends, dt, n_iter, n_coarse_sweeps, n_pred, st);
    auto key = std::make_tuple(u0, ends, dt, n_iter, n_coarse_sweeps, n_pred);
    auto it = pf->graphs.find(key);
    if (it == pf->graphs.end()) {
        cudaGraphExec_t ex = nullptr;
        MLSDC_CUDA(cudaStreamBeginCapture(pf->cap, cudaStreamCaptureModeThreadLocal));
        mlsdc_status s = pfasst_enqueue(pf, u0, ends, dt, n_iter, n_coarse_sweeps, n_pred, pf->cap);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(pf->cap, &g);
        if (s != MLSDC_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            set_error("pfasst_step graph", e);
            return MLSDC_ERR_CUDA;
        }
        it = pf->graphs.emplace(key, ex).first;
    }
    MLSDC_CUDA(cudaGraphLaunch(it->second, st));
    return MLSDC_OK;
}

extern "C" mlsdc_status pfasst_launch_count(pfasst_t pf, int64_t* launches) {
    if (!pf || !launches) return MLSDC_ERR_INVALID;
    *launches = pf->launches;
    return MLSDC_OK;
}
