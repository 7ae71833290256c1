// C ABI of the m2s library: grid hierarchy, multigrid V-cycle and PCG
// drivers (paper Sec. 7.1 HPCG: PCG with a multigrid preconditioner whose
// smoother is symmetric Gauss-Seidel; Sec. 4.3 routines), and the entry
// points declared in include/m2s.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "m2s_block.cuh"
#include "m2s_internal.cuh"
#include "m2s_pcg.cuh"
#include <nvtx3/nvToolsExt.h>

namespace {
// An NVTX range around a public call, for timelines taken under a profiler
// (a no-op when none is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace
#define M2S_RANGE(name) NvtxRange m2s_nvtx_range_(name)

using namespace m2s;

namespace {

constexpr int kMaxLevels = 8;
constexpr int kMaxTimed = 16384;  // recorded sweep launches per level

template <typename T>
struct Work {
    std::vector<T*> Qa, Qb, rc, zc;  // per level, packed over problems
    // 27-point operator: the level's right-hand side / 26 (its sweeps take
    // pre-scaled sums); NULL for the other operators
    std::vector<T*> rs;
};

}  // namespace

struct m2s_grid {
    int np = 0;
    m2s_op op = M2S_OP_HPCG27;
    int levels = 1;
    m2s_dtype pdtype = M2S_F64;
    bool has32 = false;
    std::vector<std::vector<Dims>> dims;  // [problem][level]
    std::vector<i64> ltot;                // packed points per level
    // variable-kappa hierarchy (packed per level)
    std::vector<double*> kappa;
    std::vector<KappaLevel<double>> k64;
    std::vector<KappaLevel<float>> k32;
    // sweep schedules per level, all problems in one launch (one set per dtype)
    std::vector<WaveUnits> units;
    std::vector<WaveUnits> units32;
    // batched element kernels: per level the problems' dims and chunk prefix
    std::vector<Batch> batch;
    // prefix (np + 1) of the per-problem partials of the fused p-update +
    // SpMV + p.Ap of the 27-point operator (one launch per problem)
    int* d_st27pre = nullptr;
    std::vector<int> h_st27pre;
    Work<double> w64;
    Work<float> w32;
    // PCG state (finest level, packed)
    double *r = nullptr, *z = nullptr, *zold = nullptr, *p0 = nullptr, *p1 = nullptr, *q = nullptr;
    double *z_base = nullptr, *zold_base = nullptr;  // z / zold at the start of every solve
    float *r32 = nullptr, *z32 = nullptr;
    double *part = nullptr, *part2 = nullptr;
    int npart = 0;
    PcgDev* dev = nullptr;   // one per problem
    double* x_cur = nullptr;  // solution vector of the solve in progress
    double* hist = nullptr;  // per problem: hist_cap + 1 residual norms
    int hist_cap = 0;
    DevStatus* status = nullptr;
    long long spin_ns = 4000000000LL;
    int publish_every = 4;
    int stall_level = -1;  // test hook consumed by the next sweep on that level
    int stall_unit = -1;
    BlockOp blk;
    // per-level event pairs bracketing sweep launches (m2s_sweep_timing)
    struct Timing {
        std::vector<cudaEvent_t> ev;  // 2 per recorded launch
        int used = 0, dropped = 0;
    };
    bool timing = false;
    std::vector<Timing> tim;
    // CUDA graphs of one PCG iteration (k even, k odd >= 3), captured for
    // the solution vector x_graph and replayed while it stays the same
    bool use_graphs = true;
    cudaStream_t cap_stream = nullptr;  // records the graphs (capture is not
                                        // allowed on the legacy default stream)
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    double* x_graph = nullptr;
    int graph_launches = 0;  // iterations replayed from a graph (statistics)
    std::vector<void*> allocs;
    cudaStream_t last_stream = nullptr;
    // workspaces made at first use, so that a grid used only for FP64
    // sweeps holds no Krylov vectors and no FP32 hierarchy (a 1536^3 FP64
    // vector is 29 GB)
    // ILU(0) factors of the finest level (m2s_ilu0_setup)
    double* ilu_F = nullptr;
    double* ilu_inv = nullptr;  // 1 / pivot per point
    // the application's weight records (forward, backward) and wavefront units
    double* ilu_Lw = nullptr;
    double* ilu_Uw = nullptr;
    WaveUnits ilu_units{};
    int ilu_stall_unit = -1;  // test hook consumed by the next ILU(0) application
    bool pcg_ready = false;  // r, z, zold, p0, p1, q
    bool f32_ready = false;  // FP32 level arrays, sweep schedules, r32, z32
    std::vector<int> w32_choice;  // 27-point FP32 warps per unit, per level
};

namespace {

m2s_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return M2S_OK;
    if (e == cudaErrorMemoryAllocation) {
        // a failed allocation leaves the context usable but is also kept as
        // the runtime's last error, which the next launch check would report
        cudaGetLastError();
        return M2S_ERR_OOM;
    }
    return M2S_ERR_CUDA;
}

#define M2S_TRY(expr)                                  \
    do {                                               \
        cudaError_t e__ = (expr);                      \
        if (e__ != cudaSuccess) return cuda_status(e__); \
    } while (0)

template <typename T>
cudaError_t galloc(m2s_grid* g, T** p, i64 count) {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, (size_t)std::max<i64>(count, 1) * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();  // not left behind for the next launch check
        return e;
    }
    g->allocs.push_back(v);
    *p = (T*)v;
    return cudaSuccess;
}

void destroy_grid(m2s_grid* g) {
    if (!g) return;
    cudaDeviceSynchronize();
    for (auto& u : g->units) free_wave_units(&u);
    for (auto& u : g->units32) free_wave_units(&u);
    block_free_units(&g->blk);
    for (void* p : g->allocs) cudaFree(p);
    for (auto& t : g->tim)
        for (cudaEvent_t e : t.ev) cudaEventDestroy(e);
    for (cudaGraphExec_t& ge : g->graph)
        if (ge) cudaGraphExecDestroy(ge);
    free_wave_units(&g->ilu_units);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    delete g;
}

inline cudaStream_t S(void* s) { return (cudaStream_t)s; }

// Work set of the dtype of a call.
template <typename T> Work<T>& work(m2s_grid* g);
template <> Work<double>& work<double>(m2s_grid* g) { return g->w64; }
template <> Work<float>& work<float>(m2s_grid* g) { return g->w32; }
template <typename T> const KappaLevel<T>& klev(m2s_grid* g, int l);
template <> const KappaLevel<double>& klev<double>(m2s_grid* g, int l) { return g->k64[l]; }
template <> const KappaLevel<float>& klev<float>(m2s_grid* g, int l) { return g->k32[l]; }

WaveCall wave_call(m2s_grid* g, int rev, double* rz) {
    WaveCall c;
    c.stall_unit = -1;
    c.rev = rev;
    c.publish_every = g->publish_every;
    c.spin_ns = g->spin_ns;
    c.status = g->status;
    c.rz_partials = rz;
    return c;
}

// Dims of every problem on level l.
std::vector<Dims> level_dims(m2s_grid* g, int l) {
    std::vector<Dims> v(g->np);
    for (int i = 0; i < g->np; ++i) v[i] = g->dims[i][l];
    return v;
}

// (Re)build the 27-point sweep schedules of level l: FP64 now, FP32 now if
// the FP32 hierarchy exists, else when it is made (with w32 warps).
cudaError_t build_level_units27(m2s_grid* g, int l, int w64, int w32) {
    WaveUnits a{}, b{};
    const std::vector<Dims> dl = level_dims(g, l);
    cudaError_t e = build_cta_units<double>(dl, w64, &a);
    if (e != cudaSuccess) {
        free_wave_units(&a);
        return e;
    }
    if (g->f32_ready && (e = build_cta_units<float>(dl, w32, &b)) != cudaSuccess) {
        free_wave_units(&a);
        free_wave_units(&b);
        return e;
    }
    free_wave_units(&g->units[l]);
    g->units[l] = a;
    if (g->f32_ready) {
        free_wave_units(&g->units32[l]);
        g->units32[l] = b;
    }
    g->w32_choice[l] = w32;
    return cudaSuccess;
}

// FP32 preconditioner workspaces of the 27-point operator (its level arrays
// and sweep schedules) and the finest-level r32, z32 of any operator.
cudaError_t ensure_f32(m2s_grid* g) {
    if (g->f32_ready) return cudaSuccess;
    if (!g->has32) return cudaErrorInvalidValue;
    cudaError_t e;
    if (g->op == M2S_OP_HPCG27) {
        Work<float>& w = g->w32;
        w.rs.assign(g->levels, nullptr);
        for (int l = 0; l < g->levels; ++l) {
            if ((e = galloc(g, &w.Qa[l], g->ltot[l])) != cudaSuccess ||
                (e = galloc(g, &w.Qb[l], g->ltot[l])) != cudaSuccess ||
                (e = galloc(g, &w.rs[l], g->ltot[l])) != cudaSuccess)
                return e;
            if (l > 0 && ((e = galloc(g, &w.rc[l], g->ltot[l])) != cudaSuccess ||
                          (e = galloc(g, &w.zc[l], g->ltot[l])) != cudaSuccess))
                return e;
        }
        for (int l = 0; l < g->levels; ++l) {
            WaveUnits b{};
            if ((e = build_cta_units<float>(level_dims(g, l), g->w32_choice[l], &b)) != cudaSuccess) {
                free_wave_units(&b);
                return e;
            }
            free_wave_units(&g->units32[l]);
            g->units32[l] = b;
        }
    }
    if ((e = galloc(g, &g->r32, g->ltot[0])) != cudaSuccess ||
        (e = galloc(g, &g->z32, g->ltot[0])) != cudaSuccess)
        return e;
    g->f32_ready = true;
    return cudaSuccess;
}

// Krylov vectors of the finest level (PCG and the adjoint solve).
cudaError_t ensure_pcg(m2s_grid* g) {
    cudaError_t e;
    if (!g->pcg_ready) {
        for (double** p : {&g->r, &g->z, &g->zold, &g->p0, &g->p1, &g->q})
            if ((e = galloc(g, p, g->ltot[0])) != cudaSuccess) return e;
        g->z_base = g->z;
        g->zold_base = g->zold;
        g->pcg_ready = true;
    }
    if (g->pdtype == M2S_F32 && (e = ensure_f32(g)) != cudaSuccess) return e;
    return cudaSuccess;
}

Dims coarse_of(m2s_grid* g, int i, int l) {
    return (l + 1 < g->levels) ? g->dims[i][l + 1]
                               : Dims{(g->dims[i][l].nx + 1) / 2, (g->dims[i][l].ny + 1) / 2,
                                      (g->dims[i][l].nz + 1) / 2, 0, 0};
}

// ---------------------------------------------------------------------------
// Operator-generic building blocks on level l, for all problems of the grid:
// the sweeps and the variable-kappa kernels are one launch each; the 27-point
// tile kernels are launched once per problem.
// ---------------------------------------------------------------------------
template <typename T>
cudaError_t op_spmv(m2s_grid* g, int l, const T* x, T* y, cudaStream_t st) {
    if (g->op == M2S_OP_HPCG27) {
        for (int i = 0; i < g->np; ++i) {
            const Dims d = g->dims[i][l];
            cudaError_t e = launch_spmv27<T>(d, x, y, &g->status->err, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    return launch_spmv7_b<T>(g->batch[l], klev<T>(g, l), x, y, st);
}

// Q = b + sum of the upper (up) or lower neighbours of (x + P xc).  The
// 27-point operator's Q is written as Q/26, and b/26 to bs when bs is not
// NULL.
template <typename T>
cudaError_t op_qinit(m2s_grid* g, int l, int up, const T* x, const T* xc, const T* b, T* Q, T* bs,
                     cudaStream_t st) {
    if (g->op == M2S_OP_HPCG27) {
        for (int i = 0; i < g->np; ++i) {
            const Dims d = g->dims[i][l];
            cudaError_t e =
                xc ? launch_st27_q26<T>(ST27_PROLONG_QUP, d, coarse_of(g, i, l), x, xc, b, Q, bs, st)
                   : launch_st27_q26<T>(up ? ST27_QUP : ST27_QLO, d, d, x, nullptr, b, Q, bs, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    return launch_qinit7_b<T>(g->batch[l], xc ? &g->batch[l + 1] : nullptr, klev<T>(g, l), up, x,
                              xc, b, Q, st);
}

template <typename T>
cudaError_t op_sweep(m2s_grid* g, int l, int rev, const T* Qin, T* Qout, const T* b, T* x,
                     double* rz, cudaStream_t st) {
    WaveCall c = wave_call(g, rev, rz);
    if (g->stall_level == l && g->stall_unit >= 0) {
        c.stall_unit = g->stall_unit;
        g->stall_level = -1;
        g->stall_unit = -1;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (g->timing) {
        m2s_grid::Timing& t = g->tim[l];
        if (t.used >= kMaxTimed) {
            ++t.dropped;
        } else {
            while ((int)t.ev.size() < 2 * (t.used + 1)) {
                cudaEvent_t e;
                cudaError_t er = cudaEventCreate(&e);
                if (er != cudaSuccess) return er;
                t.ev.push_back(e);
            }
            e0 = t.ev[2 * t.used];
            e1 = t.ev[2 * t.used + 1];
            ++t.used;
            cudaError_t er = cudaEventRecord(e0, st);
            if (er != cudaSuccess) return er;
        }
    }
    const WaveUnits& u = sizeof(T) == 8 ? g->units[l] : g->units32[l];
    cudaError_t e = g->op == M2S_OP_HPCG27
                        ? launch_gs27_cta<T>(u, c, Qin, Qout, b, x, st)
                        : launch_gs7_cta<T>(u, c, klev<T>(g, l), Qin, Qout, b, x, st);
    if (e == cudaSuccess && e1) e = cudaEventRecord(e1, st);
    return e;
}

// rc = R (r - A z); the 27-point operator also writes rc/26 to rcs when not NULL
template <typename T>
cudaError_t op_restrict(m2s_grid* g, int l, const T* r, const T* z, T* rc, T* rcs,
                        cudaStream_t st) {
    if (g->op == M2S_OP_HPCG27) {
        for (int i = 0; i < g->np; ++i) {
            cudaError_t e =
                launch_restrict27<T>(g->dims[i][l], g->dims[i][l + 1], r, z, rc, rcs, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    return launch_restrict7_b<T>(g->batch[l], g->batch[l + 1], klev<T>(g, l), r, z, rc, st);
}

// V-cycle from level l for all problems: z = M_l^-1 r (packed level-l
// arrays).  rs is r/26 for the 27-point operator (whose sweeps take Q/26 and
// write Q/26 from b/26) and r itself otherwise.  rz (optional) receives the
// b.x partials of the last sweep of the finest level, W per sweep unit.
template <typename T>
cudaError_t vcycle(m2s_grid* g, int l, const T* r, const T* rs, T* z, double* rz,
                   cudaStream_t st) {
    Work<T>& w = work<T>(g);
    T* Qa = w.Qa[l];
    T* Qb = w.Qb[l];
    cudaError_t e;
    // pre-smoothing from z = 0: the old-neighbour sum is r itself
    if ((e = op_sweep<T>(g, l, 0, rs, Qb, rs, z, nullptr, st)) != cudaSuccess) return e;
    if (l == g->levels - 1) return op_sweep<T>(g, l, 1, Qb, nullptr, r, z, rz, st);
    if ((e = op_sweep<T>(g, l, 1, Qb, nullptr, r, z, nullptr, st)) != cudaSuccess) return e;
    T* rcs = w.rs.empty() ? nullptr : w.rs[l + 1];
    if ((e = op_restrict<T>(g, l, r, z, w.rc[l + 1], rcs, st)) != cudaSuccess) return e;
    if ((e = vcycle<T>(g, l + 1, w.rc[l + 1], rcs ? rcs : w.rc[l + 1], w.zc[l + 1], nullptr, st)) !=
        cudaSuccess)
        return e;
    // prolongation fused into the old-neighbour sum of the post-smoothing
    if ((e = op_qinit<T>(g, l, 1, z, w.zc[l + 1], r, Qa, nullptr, st)) != cudaSuccess) return e;
    if ((e = op_sweep<T>(g, l, 0, Qa, Qb, rs, z, nullptr, st)) != cudaSuccess) return e;
    return op_sweep<T>(g, l, 1, Qb, nullptr, r, z, rz, st);
}

// V-cycle on a caller's r: the 27-point operator first forms r/26
template <typename T>
cudaError_t vcycle_from(m2s_grid* g, const T* r, T* z, cudaStream_t st) {
    Work<T>& w = work<T>(g);
    if (w.rs.empty()) return vcycle<T>(g, 0, r, r, z, nullptr, st);
    cudaError_t e = launch_scale26<T>(g->ltot[0], r, w.rs[0], st);
    if (e != cudaSuccess) return e;
    return vcycle<T>(g, 0, r, w.rs[0], z, nullptr, st);
}

template <typename T>
cudaError_t symgs(m2s_grid* g, int l, const T* b, T* x, int sweeps, cudaStream_t st) {
    Work<T>& w = work<T>(g);
    // sweeps that write Q take b/26 for the 27-point operator (formed by the
    // first Q kernel), b otherwise
    T* bs = w.rs.empty() ? nullptr : w.rs[l];
    const T* bq = bs ? bs : b;
    cudaError_t e;
    if ((e = op_qinit<T>(g, l, 1, x, nullptr, b, w.Qa[l], bs, st)) != cudaSuccess) return e;
    for (int s = 0; s < sweeps; ++s) {
        if ((e = op_sweep<T>(g, l, 0, w.Qa[l], w.Qb[l], bq, x, nullptr, st)) != cudaSuccess) return e;
        T* qn = (s + 1 < sweeps) ? w.Qa[l] : nullptr;
        if ((e = op_sweep<T>(g, l, 1, w.Qb[l], qn, bq, x, nullptr, st)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t gs_sweep(m2s_grid* g, int l, const T* b, T* x, int rev, cudaStream_t st) {
    Work<T>& w = work<T>(g);
    cudaError_t e;
    if ((e = op_qinit<T>(g, l, rev ? 0 : 1, x, nullptr, b, w.Qa[l], nullptr, st)) != cudaSuccess)
        return e;
    return op_sweep<T>(g, l, rev, w.Qa[l], nullptr, b, x, nullptr, st);
}

bool valid_level(m2s_grid* g, int level) { return g && level >= 0 && level < g->levels; }

// FP64 always; FP32 where the grid has an FP32 hierarchy (made on first use)
m2s_status check_dtype(m2s_grid* g, m2s_dtype dt) {
    if (dt == M2S_F64) return M2S_OK;
    if (dt != M2S_F32 || !g->has32) return M2S_ERR_INVALID_ARG;
    return cuda_status(ensure_f32(g));
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

// ---------------------------------------------------------------------------
// PCG for all problems of the grid at once (finest level, packed): x0 = 0,
// r0 = b, per-problem scalars; a problem that reaches its tolerance is
// frozen on the device while the others iterate.
// ---------------------------------------------------------------------------
cudaError_t pcg_iteration(m2s_grid* g, int k, cudaStream_t st) {
    const Batch& b0 = g->batch[0];
    const int np = g->np;
    const i64 n = g->ltot[0];
    const int stride = g->hist_cap + 1;
    cudaError_t e;
    // z = M^-1 r and rho = r.z
    if (g->pdtype == M2S_F32) {
        float* r32s = g->w32.rs.empty() ? nullptr : g->w32.rs[0];
        if ((e = launch_cast_down(n, g->r, g->r32, r32s, st)) != cudaSuccess) return e;
        if ((e = vcycle<float>(g, 0, g->r32, r32s ? r32s : g->r32, g->z32, nullptr, st)) !=
            cudaSuccess)
            return e;
        double* zo = (k > 1) ? g->zold : nullptr;
        if ((e = launch_cast_up_dots_b(b0, g->z32, g->r, zo, g->z, g->part, g->part2, st)) !=
            cudaSuccess)
            return e;
        if ((e = launch_finalize_b(FIN_RHO, g->dev, np, g->part, b0.cstart, zo ? g->part2 : nullptr,
                                   b0.cstart, nullptr, stride, 0.0, 0, st)) != cudaSuccess)
            return e;
    } else {
        const double* rs = g->w64.rs.empty() ? g->r : g->w64.rs[0];
        if ((e = vcycle<double>(g, 0, g->r, rs, g->z, g->part, st)) != cudaSuccess) return e;
        if ((e = launch_finalize_b(FIN_RHO, g->dev, np, g->part, g->units[0].d_rzpre, nullptr,
                                   nullptr, nullptr, stride, 0.0, 0, st)) != cudaSuccess)
            return e;
    }
    // p = z + beta p; q = A p; p.q   (p ping-pongs between p0 and p1)
    double* pin = (k & 1) ? g->p1 : g->p0;
    double* pout = (k & 1) ? g->p0 : g->p1;
    if (g->op == M2S_OP_HPCG27) {
        for (int i = 0; i < np; ++i) {
            const double* beta = (k == 1) ? nullptr : &g->dev[i].beta;
            if ((e = launch_pspmv_dot(g->dims[i][0], g->z, pin, pout, g->q, beta,
                                      g->part + g->h_st27pre[i], &g->status->err, st)) !=
                cudaSuccess)
                return e;
        }
        if ((e = launch_finalize_b(FIN_PQ, g->dev, np, g->part, g->d_st27pre, nullptr, nullptr,
                                   nullptr, stride, 0.0, 0, st)) != cudaSuccess)
            return e;
    } else {
        if ((e = launch_paxpy_b(b0, g->dev, k == 1, g->z, pin, pout, st)) != cudaSuccess) return e;
        if ((e = op_spmv<double>(g, 0, pout, g->q, st)) != cudaSuccess) return e;
        if ((e = launch_dot_b<double>(b0, pout, g->q, g->part, st)) != cudaSuccess) return e;
        if ((e = launch_finalize_b(FIN_PQ, g->dev, np, g->part, b0.cstart, nullptr, nullptr,
                                   nullptr, stride, 0.0, 0, st)) != cudaSuccess)
            return e;
    }
    // r/26 for the FP64 V-cycle of the 27-point operator
    double* rs = (g->pdtype == M2S_F64 && !g->w64.rs.empty()) ? g->w64.rs[0] : nullptr;
    if ((e = launch_update_b(b0, g->dev, pout, g->q, g->x_cur, g->r, rs, g->part, st)) !=
        cudaSuccess)
        return e;
    if ((e = launch_finalize_b(FIN_RR, g->dev, np, g->part, b0.cstart, nullptr, nullptr, g->hist,
                               stride, 0.0, 0, st)) != cudaSuccess)
        return e;
    if (g->pdtype == M2S_F32) std::swap(g->z, g->zold);
    return cudaSuccess;
}

m2s_status pcg_batch(m2s_grid* g, const double* b, double* x, const m2s_pcg_opts& o,
                     m2s_pcg_result* out, cudaStream_t st) {
    const Batch& b0 = g->batch[0];
    const int np = g->np;
    const i64 n = g->ltot[0];
    const int stride = g->hist_cap + 1;
    g->x_cur = x;
    // the FP32 form swaps z and zold every iteration: start from the same
    // assignment in every solve (the captured graphs rely on it)
    g->z = g->z_base;
    g->zold = g->zold_base;
    M2S_TRY(cudaMemsetAsync(x, 0, n * sizeof(double), st));
    M2S_TRY(cudaMemcpyAsync(g->r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (g->pdtype == M2S_F64 && !g->w64.rs.empty())
        M2S_TRY(launch_scale26<double>(n, g->r, g->w64.rs[0], st));
    M2S_TRY(launch_dot_b<double>(b0, g->r, g->r, g->part, st));
    M2S_TRY(launch_finalize_b(FIN_BB, g->dev, np, g->part, b0.cstart, nullptr, nullptr, g->hist,
                              stride, o.rtol * o.rtol, o.fixed_iters ? 1 : 0, st));
    std::vector<PcgDev> h(np);
    // graphs are replayed only when nothing host-side varies between
    // iterations of the same parity: no per-launch timing, no pending stall
    const bool graphs = g->use_graphs && !g->timing && g->stall_unit < 0;
    if (!graphs || g->x_graph != x) {
        for (cudaGraphExec_t& ge : g->graph)
            if (ge) cudaGraphExecDestroy(ge), ge = nullptr;
        g->x_graph = nullptr;
    }
    for (int k = 1; k <= o.max_iters; ++k) {
        if (graphs && k >= 2) {
            cudaGraphExec_t& ge = g->graph[k & 1];
            if (!ge) {
                // record this iteration once on the grid's own stream (its
                // launches are recorded, not run), then replay it on st
                cudaGraph_t gr = nullptr;
                if (!g->cap_stream)
                    M2S_TRY(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
                M2S_TRY(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
                const cudaError_t ce = pcg_iteration(g, k, g->cap_stream);
                const cudaError_t ee = cudaStreamEndCapture(g->cap_stream, &gr);
                if (ce != cudaSuccess || ee != cudaSuccess) {
                    if (gr) cudaGraphDestroy(gr);
                    return cuda_status(ce != cudaSuccess ? ce : ee);
                }
                const cudaError_t ie = cudaGraphInstantiate(&ge, gr, 0);
                cudaGraphDestroy(gr);
                if (ie != cudaSuccess) {
                    ge = nullptr;
                    return cuda_status(ie);
                }
                g->x_graph = x;
            } else if (g->pdtype == M2S_F32) {
                std::swap(g->z, g->zold);  // the host-side state a run would leave
            }
            M2S_TRY(cudaGraphLaunch(ge, st));
            ++g->graph_launches;
        } else {
            M2S_TRY(pcg_iteration(g, k, st));
        }
        const bool last = k == o.max_iters;
        if (!o.fixed_iters && (k % o.check_every == 0 || last)) {
            M2S_TRY(cudaMemcpyAsync(h.data(), g->dev, np * sizeof(PcgDev), cudaMemcpyDeviceToHost,
                                    st));
            M2S_TRY(cudaStreamSynchronize(st));
            bool all_done = true, bad = false;
            for (const PcgDev& s : h) {
                all_done = all_done && s.done;
                bad = bad || s.status != 0;
            }
            if (all_done || bad) break;
        }
    }
    M2S_TRY(cudaMemcpyAsync(h.data(), g->dev, np * sizeof(PcgDev), cudaMemcpyDeviceToHost, st));
    M2S_TRY(cudaStreamSynchronize(st));
    DevStatus ds;
    M2S_TRY(cudaMemcpy(&ds, g->status, sizeof(DevStatus), cudaMemcpyDeviceToHost));
    if (ds.err != 0) {
        cudaMemset(g->status, 0, sizeof(DevStatus));
        return (m2s_status)ds.err;
    }
    bool bad = false, all_done = true;
    if (out) {
        out->iters = 0;
        out->rel_resid = 0.0;
        out->resid_hist_last = 0.0;
    }
    for (const PcgDev& s : h) {
        bad = bad || s.status != 0;
        all_done = all_done && (s.done || !(s.bb > 0));
        if (out) {
            out->iters = std::max(out->iters, s.iter);
            out->resid_hist_last = std::max(out->resid_hist_last, std::sqrt(s.rr));
            out->rel_resid = std::max(out->rel_resid, s.bb > 0 ? std::sqrt(s.rr / s.bb) : 0.0);
        }
    }
    if (bad) return M2S_ERR_BREAKDOWN;
    if (!o.fixed_iters && !all_done) return M2S_ERR_NOT_CONVERGED;
    return M2S_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* m2s_status_string(m2s_status s) {
    switch (s) {
        case M2S_OK: return "ok";
        case M2S_ERR_INVALID_ARG: return "invalid argument";
        case M2S_ERR_CUDA: return "CUDA error";
        case M2S_ERR_OOM: return "out of device memory";
        case M2S_ERR_TIMEOUT: return "a bounded spin-wait expired";
        case M2S_ERR_NOT_CONVERGED: return "not converged";
        case M2S_ERR_BREAKDOWN: return "breakdown (non-finite value or p.Ap <= 0)";
    }
    return "unknown status";
}

static bool is_block(m2s_op op) { return op == M2S_OP_BLOCK7_5x5 || op == M2S_OP_BLOCK7_JAC; }

m2s_status m2s_grid_create(const m2s_grid_desc* descs, int n_problems, void* stream,
                           m2s_grid** out) {
    M2S_RANGE("m2s_grid_create");
    if (!out) return M2S_ERR_INVALID_ARG;
    *out = nullptr;
    if (!descs || n_problems < 1) return M2S_ERR_INVALID_ARG;
    const m2s_op op = descs[0].op;
    const int levels = descs[0].mg_levels;
    const m2s_dtype pdt = descs[0].precond_dtype;
    if (op != M2S_OP_HPCG27 && op != M2S_OP_DIFF7_KAPPA && !is_block(op)) return M2S_ERR_INVALID_ARG;
    if (levels < 1 || levels > kMaxLevels) return M2S_ERR_INVALID_ARG;
    if (pdt != M2S_F64 && pdt != M2S_F32) return M2S_ERR_INVALID_ARG;
    for (int i = 0; i < n_problems; ++i) {
        const m2s_grid_desc& d = descs[i];
        if (d.op != op || d.mg_levels != levels || d.precond_dtype != pdt) return M2S_ERR_INVALID_ARG;
        if (d.nx < 1 || d.ny < 1 || d.nz < 1) return M2S_ERR_INVALID_ARG;
        if ((i64)d.nx * d.ny * d.nz > (1LL << 34)) return M2S_ERR_INVALID_ARG;
        if (op == M2S_OP_DIFF7_KAPPA && (!d.kappa || !aligned(d.kappa, 8))) return M2S_ERR_INVALID_ARG;
        if (op == M2S_OP_BLOCK7_5x5 && (!d.D || !d.L || !d.U)) return M2S_ERR_INVALID_ARG;
        if (op == M2S_OP_BLOCK7_JAC && !d.jac) return M2S_ERR_INVALID_ARG;
    }
    cudaStream_t st = S(stream);
    m2s_grid* g = new (std::nothrow) m2s_grid();
    if (!g) return M2S_ERR_OOM;
    g->np = n_problems;
    g->op = op;
    g->levels = is_block(op) ? 1 : levels;
    g->pdtype = pdt;
    g->has32 = op == M2S_OP_HPCG27 || (op == M2S_OP_DIFF7_KAPPA && pdt == M2S_F32);
    const int L = g->levels;
    g->tim.resize(L);
    g->dims.assign(n_problems, std::vector<Dims>(L));
    g->ltot.assign(L, 0);
    for (int l = 0; l < L; ++l)
        for (int i = 0; i < n_problems; ++i) {
            Dims d;
            if (l == 0) {
                d.nx = descs[i].nx;
                d.ny = descs[i].ny;
                d.nz = descs[i].nz;
            } else {
                const Dims& f = g->dims[i][l - 1];
                d.nx = (f.nx + 1) / 2;
                d.ny = (f.ny + 1) / 2;
                d.nz = (f.nz + 1) / 2;
            }
            d.n = (i64)d.nx * d.ny * d.nz;
            d.off = g->ltot[l];
            g->ltot[l] += d.n;
            g->dims[i][l] = d;
        }
    auto fail = [&](cudaError_t e) {
        destroy_grid(g);
        return cuda_status(e);
    };
    cudaError_t e = cudaSuccess;
    if ((e = galloc(g, &g->status, 1)) != cudaSuccess) return fail(e);
    if ((e = cudaMemsetAsync(g->status, 0, sizeof(DevStatus), st)) != cudaSuccess) return fail(e);
    if ((e = galloc(g, &g->dev, n_problems)) != cudaSuccess) return fail(e);
    if ((e = cudaMemsetAsync(g->dev, 0, n_problems * sizeof(PcgDev), st)) != cudaSuccess)
        return fail(e);

    if (is_block(op)) {
        e = block_create(&g->blk, descs, n_problems, g->dims, st,
                         [g](void** p, size_t bytes) -> cudaError_t {
                             cudaError_t ee = cudaMalloc(p, bytes);
                             if (ee == cudaSuccess) g->allocs.push_back(*p);
                             return ee;
                         });
        if (e != cudaSuccess) return fail(e);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e);
        *out = g;
        return M2S_OK;
    }

    // workspaces per level
    g->w64.Qa.assign(L, nullptr); g->w64.Qb.assign(L, nullptr);
    g->w64.rc.assign(L, nullptr); g->w64.zc.assign(L, nullptr);
    g->w32.Qa.assign(L, nullptr); g->w32.Qb.assign(L, nullptr);
    g->w32.rc.assign(L, nullptr); g->w32.zc.assign(L, nullptr);
    if (op == M2S_OP_HPCG27) g->w64.rs.assign(L, nullptr);
    g->w32_choice.assign(L, 8);
    for (int l = 0; l < L; ++l) {
        if (!g->w64.rs.empty() && (e = galloc(g, &g->w64.rs[l], g->ltot[l])) != cudaSuccess)
            return fail(e);
        if ((e = galloc(g, &g->w64.Qa[l], g->ltot[l])) != cudaSuccess) return fail(e);
        if ((e = galloc(g, &g->w64.Qb[l], g->ltot[l])) != cudaSuccess) return fail(e);
        if (l > 0) {
            if ((e = galloc(g, &g->w64.rc[l], g->ltot[l])) != cudaSuccess) return fail(e);
            if ((e = galloc(g, &g->w64.zc[l], g->ltot[l])) != cudaSuccess) return fail(e);
        }
        // the 27-point operator's FP32 arrays are made at first FP32 use
        if (g->has32 && op != M2S_OP_HPCG27) {
            if ((e = galloc(g, &g->w32.Qa[l], g->ltot[l])) != cudaSuccess) return fail(e);
            if ((e = galloc(g, &g->w32.Qb[l], g->ltot[l])) != cudaSuccess) return fail(e);
            if (l > 0) {
                if ((e = galloc(g, &g->w32.rc[l], g->ltot[l])) != cudaSuccess) return fail(e);
                if ((e = galloc(g, &g->w32.zc[l], g->ltot[l])) != cudaSuccess) return fail(e);
            }
        }
    }
    // kappa hierarchy
    if (op == M2S_OP_DIFF7_KAPPA) {
        g->kappa.assign(L, nullptr);
        g->k64.resize(L);
        g->k32.resize(L);
        for (int l = 0; l < L; ++l) {
            if ((e = galloc(g, &g->kappa[l], g->ltot[l])) != cudaSuccess) return fail(e);
            KappaLevel<double>& k = g->k64[l];
            for (int c = 0; c < 3; ++c)
                if ((e = galloc(g, &k.kf[c], g->ltot[l])) != cudaSuccess ||
                    (e = galloc(g, &k.kr[c], g->ltot[l])) != cudaSuccess)
                    return fail(e);
            if ((e = galloc(g, &k.diag, g->ltot[l])) != cudaSuccess) return fail(e);
            if ((e = galloc(g, &k.invdiag, g->ltot[l])) != cudaSuccess) return fail(e);
            for (int c = 0; c < 2; ++c)
                if ((e = galloc(g, &k.pack[c], 4 * g->ltot[l])) != cudaSuccess) return fail(e);
            if (g->has32) {
                KappaLevel<float>& k3 = g->k32[l];
                for (int c = 0; c < 3; ++c)
                    if ((e = galloc(g, &k3.kf[c], g->ltot[l])) != cudaSuccess ||
                        (e = galloc(g, &k3.kr[c], g->ltot[l])) != cudaSuccess)
                        return fail(e);
                if ((e = galloc(g, &k3.diag, g->ltot[l])) != cudaSuccess) return fail(e);
                if ((e = galloc(g, &k3.invdiag, g->ltot[l])) != cudaSuccess) return fail(e);
                for (int c = 0; c < 2; ++c)
                    if ((e = galloc(g, &k3.pack[c], 4 * g->ltot[l])) != cudaSuccess) return fail(e);
            }
        }
        for (int i = 0; i < n_problems; ++i) {
            const Dims& d = g->dims[i][0];
            if ((e = cudaMemcpyAsync(g->kappa[0] + d.off, descs[i].kappa, d.n * sizeof(double),
                                     cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
                return fail(e);
            for (int l = 1; l < L; ++l)
                if ((e = launch_kappa_coarsen(g->dims[i][l - 1], g->dims[i][l], g->kappa[l - 1],
                                              g->kappa[l], st)) != cudaSuccess)
                    return fail(e);
            for (int l = 0; l < L; ++l) {
                if ((e = launch_kappa_setup<double>(g->dims[i][l], g->kappa[l], g->k64[l], st)) !=
                    cudaSuccess)
                    return fail(e);
                if (g->has32 &&
                    (e = launch_kappa_setup<float>(g->dims[i][l], g->kappa[l], g->k32[l], st)) !=
                        cudaSuccess)
                    return fail(e);
            }
        }
    }
    // batched element kernels: per level the problems' dims and chunk prefix
    g->batch.assign(L, Batch{});
    for (int l = 0; l < L; ++l) {
        std::vector<Dims> dl = level_dims(g, l);
        std::vector<int> cs(n_problems + 1, 0);
        for (int i = 0; i < n_problems; ++i)
            cs[i + 1] = cs[i] + (int)((dl[i].n + kChunk - 1) / kChunk);
        Dims* dd = nullptr;
        int* dc = nullptr;
        if ((e = galloc(g, &dd, n_problems)) != cudaSuccess ||
            (e = galloc(g, &dc, n_problems + 1)) != cudaSuccess ||
            (e = cudaMemcpy(dd, dl.data(), n_problems * sizeof(Dims), cudaMemcpyHostToDevice)) !=
                cudaSuccess ||
            (e = cudaMemcpy(dc, cs.data(), (n_problems + 1) * sizeof(int),
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return fail(e);
        g->batch[l] = Batch{n_problems, dd, dc, cs.back()};
    }
    // sweep schedules, one unit table per level and dtype for all problems
    g->units.assign(L, WaveUnits{});
    g->units32.assign(L, WaveUnits{});
    for (int l = 0; l < L; ++l) {
        if (op == M2S_OP_HPCG27) {
            const std::vector<Dims> dl = level_dims(g, l);
            if ((e = build_level_units27(g, l, cta_default_warps(1, dl), cta_default_warps(0, dl))) !=
                cudaSuccess)
                return fail(e);
        } else {
            if ((e = build_cta7_units<double>(level_dims(g, l), &g->units[l])) != cudaSuccess)
                return fail(e);
            if (g->has32 &&
                (e = build_cta7_units<float>(level_dims(g, l), &g->units32[l])) != cudaSuccess)
                return fail(e);
        }
    }
    // the variable-kappa operator's FP32 hierarchy is made with its
    // coefficients above; its r32, z32 and every PCG vector at first use
    // partial sums: chunks of the finest level, the 27-point fused SpMV's
    // tiles of every problem, or the b.x partials of any sweep schedule
    g->h_st27pre.assign(n_problems + 1, 0);
    for (int i = 0; i < n_problems; ++i)
        g->h_st27pre[i + 1] = g->h_st27pre[i] + st27_num_partials(g->dims[i][0]);
    if ((e = galloc(g, &g->d_st27pre, n_problems + 1)) != cudaSuccess ||
        (e = cudaMemcpy(g->d_st27pre, g->h_st27pre.data(), (n_problems + 1) * sizeof(int),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e);
    int np = std::max(g->batch[0].nchunks, g->h_st27pre.back());
    np = std::max(np, op == M2S_OP_HPCG27 ? cta_rz_partials_max(level_dims(g, 0))
                                          : g->units[0].n_rz);
    g->npart = np;
    if ((e = galloc(g, &g->part, np)) != cudaSuccess) return fail(e);
    if ((e = galloc(g, &g->part2, np)) != cudaSuccess) return fail(e);
    g->hist_cap = 4096;
    if ((e = galloc(g, &g->hist, (i64)(g->hist_cap + 1) * n_problems)) != cudaSuccess)
        return fail(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e);
    *out = g;
    return M2S_OK;
}

m2s_status m2s_grid_destroy(m2s_grid* grid) {
    destroy_grid(grid);
    return M2S_OK;
}

m2s_status m2s_debug_stall_unit(m2s_grid* grid, int level, int unit) {
    if (!grid || unit < 0 || is_block(grid->op)) return M2S_ERR_INVALID_ARG;
    if (level == -1) {  // the next ILU(0) application's forward substitution
        if (grid->op != M2S_OP_HPCG27) return M2S_ERR_INVALID_ARG;
        grid->ilu_stall_unit = unit;
        return M2S_OK;
    }
    if (!valid_level(grid, level)) return M2S_ERR_INVALID_ARG;
    grid->stall_level = level;
    grid->stall_unit = unit;
    return M2S_OK;
}

m2s_status m2s_sweep_timing(m2s_grid* grid, int enable) {
    if (!grid) return M2S_ERR_INVALID_ARG;
    if (enable)
        for (auto& t : grid->tim) t.used = t.dropped = 0;
    grid->timing = enable != 0;
    return M2S_OK;
}

m2s_status m2s_sweep_timing_read(m2s_grid* grid, int level, int* launches, double* total_ms,
                                 int* dropped) {
    if (!grid || level < 0 || level >= (int)grid->tim.size()) return M2S_ERR_INVALID_ARG;
    const m2s_grid::Timing& t = grid->tim[level];
    double ms = 0.0;
    for (int k = 0; k < t.used; ++k) {
        M2S_TRY(cudaEventSynchronize(t.ev[2 * k + 1]));
        float f = 0.f;
        M2S_TRY(cudaEventElapsedTime(&f, t.ev[2 * k], t.ev[2 * k + 1]));
        ms += f;
    }
    if (launches) *launches = t.used;
    if (total_ms) *total_ms = ms;
    if (dropped) *dropped = t.dropped;
    return M2S_OK;
}

m2s_status m2s_sweep_warps(m2s_grid* grid, int level, int* warps_f64, int* warps_f32) {
    if (!grid || !warps_f64 || !warps_f32 || grid->op != M2S_OP_HPCG27) return M2S_ERR_INVALID_ARG;
    if (level < 0 || level >= grid->levels) return M2S_ERR_INVALID_ARG;
    *warps_f64 = grid->units[level].W;
    *warps_f32 = grid->w32_choice[level];
    return M2S_OK;
}

m2s_status m2s_set_sweep_warps(m2s_grid* grid, int level, int warps) {
    if (!grid || grid->op != M2S_OP_HPCG27 || !cta_warps_supported(warps)) return M2S_ERR_INVALID_ARG;
    if (level < -1 || level >= grid->levels) return M2S_ERR_INVALID_ARG;
    M2S_TRY(cudaDeviceSynchronize());
    for (int l = 0; l < grid->levels; ++l) {
        if (level >= 0 && l != level) continue;
        M2S_TRY(build_level_units27(grid, l, warps, warps));
    }
    return M2S_OK;
}

m2s_status m2s_autotune_sweeps(m2s_grid* g, int reps, void* stream, int* chosen) {
    M2S_RANGE("m2s_autotune_sweeps");
    if (!g || g->op != M2S_OP_HPCG27 || reps < 1) return M2S_ERR_INVALID_ARG;
    M2S_TRY(ensure_f32(g));
    cudaStream_t st = S(stream);
    cudaEvent_t e0, e1;
    M2S_TRY(cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_status(e);
    }
    const bool timing = g->timing;
    g->timing = false;
    // scratch: the level's own work vectors (their contents are not kept
    // between calls; on the finest level the r/26 and second Q buffers);
    // b = 0 and x = 0, so the sweeps compute zeros
    auto time_sweeps = [&](int l, bool f64, float* ms) -> cudaError_t {
        const i64 n = g->ltot[l];
        cudaError_t er;
        if (f64) {
            double* b = l == 0 ? g->w64.rs[0] : g->w64.rc[l];
            double* x = l == 0 ? g->w64.Qb[0] : g->w64.zc[l];
            if ((er = cudaMemsetAsync(b, 0, n * sizeof(double), st)) != cudaSuccess ||
                (er = cudaMemsetAsync(x, 0, n * sizeof(double), st)) != cudaSuccess ||
                (er = gs_sweep<double>(g, l, b, x, 0, st)) != cudaSuccess ||
                (er = cudaEventRecord(e0, st)) != cudaSuccess)
                return er;
            for (int k = 0; k < reps; ++k)
                if ((er = op_sweep<double>(g, l, 0, g->w64.Qa[l], nullptr, b, x, nullptr, st)) !=
                    cudaSuccess)
                    return er;
        } else {
            float* b = l == 0 ? g->w32.rs[0] : g->w32.rc[l];
            float* x = l == 0 ? g->w32.Qb[0] : g->w32.zc[l];
            if ((er = cudaMemsetAsync(b, 0, n * sizeof(float), st)) != cudaSuccess ||
                (er = cudaMemsetAsync(x, 0, n * sizeof(float), st)) != cudaSuccess ||
                (er = gs_sweep<float>(g, l, b, x, 0, st)) != cudaSuccess ||
                (er = cudaEventRecord(e0, st)) != cudaSuccess)
                return er;
            for (int k = 0; k < reps; ++k)
                if ((er = op_sweep<float>(g, l, 0, g->w32.Qa[l], nullptr, b, x, nullptr, st)) !=
                    cudaSuccess)
                    return er;
        }
        if ((er = cudaEventRecord(e1, st)) != cudaSuccess ||
            (er = cudaEventSynchronize(e1)) != cudaSuccess)
            return er;
        return cudaEventElapsedTime(ms, e0, e1);
    };
    for (int l = 0; l < g->levels && e == cudaSuccess; ++l) {
        int best[2] = {8, 8};
        float best_ms[2] = {1e30f, 1e30f};
        for (int w : {4, 8}) {
            if ((e = build_level_units27(g, l, w, w)) != cudaSuccess) break;
            for (int f = 0; f < 2 && e == cudaSuccess; ++f) {
                float ms = 0.f;
                if ((e = time_sweeps(l, f == 0, &ms)) != cudaSuccess) break;
                if (ms < best_ms[f]) best_ms[f] = ms, best[f] = w;
            }
        }
        if (e == cudaSuccess) e = build_level_units27(g, l, best[0], best[1]);
        if (chosen && e == cudaSuccess) {
            chosen[2 * l] = best[0];
            chosen[2 * l + 1] = best[1];
        }
    }
    g->timing = timing;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_status(e);
    return m2s_grid_sync(g, stream);
}

m2s_status m2s_set_graphs(m2s_grid* grid, int enable) {
    if (!grid) return M2S_ERR_INVALID_ARG;
    grid->use_graphs = enable != 0;
    return M2S_OK;
}

m2s_status m2s_set_spin_limit(m2s_grid* grid, long long limit_ns) {
    if (!grid || limit_ns <= 0) return M2S_ERR_INVALID_ARG;
    grid->spin_ns = limit_ns;
    return M2S_OK;
}

long long m2s_grid_points(const m2s_grid* grid, int problem, int level) {
    if (!grid || problem < 0 || problem >= grid->np || level < 0 || level >= grid->levels) return 0;
    return grid->dims[problem][level].n;
}

m2s_status m2s_grid_sync(m2s_grid* grid, void* stream) {
    if (!grid) return M2S_ERR_INVALID_ARG;
    M2S_TRY(cudaStreamSynchronize(S(stream)));
    DevStatus ds;
    M2S_TRY(cudaMemcpy(&ds, grid->status, sizeof(DevStatus), cudaMemcpyDeviceToHost));
    if (ds.err != 0) {
        M2S_TRY(cudaMemset(grid->status, 0, sizeof(DevStatus)));
        return (m2s_status)ds.err;
    }
    return M2S_OK;
}

m2s_status m2s_spmv(m2s_grid* g, int level, m2s_dtype dtype, const void* x, void* y, void* stream) {
    M2S_RANGE("m2s_spmv");
    if (!valid_level(g, level) || !x || !y || x == y) return M2S_ERR_INVALID_ARG;
    if (is_block(g->op)) {
        if (dtype != M2S_F64) return M2S_ERR_INVALID_ARG;
        return cuda_status(block_apply(&g->blk, (const double*)x, (double*)y, S(stream)));
    }
    if (m2s_status cs = check_dtype(g, dtype)) return cs;
    if (dtype == M2S_F64) M2S_TRY(op_spmv<double>(g, level, (const double*)x, (double*)y, S(stream)));
    else M2S_TRY(op_spmv<float>(g, level, (const float*)x, (float*)y, S(stream)));
    return M2S_OK;
}

m2s_status m2s_symgs(m2s_grid* g, int level, m2s_dtype dtype, const void* b, void* x,
                     int n_sym_sweeps, void* stream) {
    M2S_RANGE("m2s_symgs");
    if (!valid_level(g, level) || !b || !x || b == x || n_sym_sweeps < 0) return M2S_ERR_INVALID_ARG;
    if (is_block(g->op)) return M2S_ERR_INVALID_ARG;
    if (m2s_status cs = check_dtype(g, dtype)) return cs;
    if (n_sym_sweeps == 0) return M2S_OK;
    if (dtype == M2S_F64)
        M2S_TRY(symgs<double>(g, level, (const double*)b, (double*)x, n_sym_sweeps, S(stream)));
    else
        M2S_TRY(symgs<float>(g, level, (const float*)b, (float*)x, n_sym_sweeps, S(stream)));
    return M2S_OK;
}

m2s_status m2s_gs_sweep(m2s_grid* g, int level, m2s_dtype dtype, const void* b, void* x,
                        m2s_direction direction, void* stream) {
    M2S_RANGE("m2s_gs_sweep");
    if (!valid_level(g, level) || !b || !x || b == x) return M2S_ERR_INVALID_ARG;
    if (direction != M2S_FORWARD && direction != M2S_BACKWARD) return M2S_ERR_INVALID_ARG;
    if (is_block(g->op)) return M2S_ERR_INVALID_ARG;
    if (m2s_status cs = check_dtype(g, dtype)) return cs;
    const int rev = direction == M2S_BACKWARD;
    if (dtype == M2S_F64)
        M2S_TRY(gs_sweep<double>(g, level, (const double*)b, (double*)x, rev, S(stream)));
    else
        M2S_TRY(gs_sweep<float>(g, level, (const float*)b, (float*)x, rev, S(stream)));
    return M2S_OK;
}

m2s_status m2s_mg_restrict(m2s_grid* g, int level, m2s_dtype dtype, const void* r, const void* z,
                           void* rc, void* stream) {
    M2S_RANGE("m2s_mg_restrict");
    if (!g || level < 0 || level + 1 >= g->levels || !r || !z || !rc) return M2S_ERR_INVALID_ARG;
    if (is_block(g->op)) return M2S_ERR_INVALID_ARG;
    if (m2s_status cs = check_dtype(g, dtype)) return cs;
    if (dtype == M2S_F64)
        M2S_TRY(op_restrict<double>(g, level, (const double*)r, (const double*)z, (double*)rc, nullptr,
                                    S(stream)));
    else
        M2S_TRY(op_restrict<float>(g, level, (const float*)r, (const float*)z, (float*)rc, nullptr,
                                   S(stream)));
    return M2S_OK;
}

m2s_status m2s_mg_prolong(m2s_grid* g, int level, m2s_dtype dtype, const void* zc, void* z,
                          void* stream) {
    M2S_RANGE("m2s_mg_prolong");
    if (!g || level < 0 || level + 1 >= g->levels || !zc || !z) return M2S_ERR_INVALID_ARG;
    if (is_block(g->op)) return M2S_ERR_INVALID_ARG;
    if (m2s_status cs = check_dtype(g, dtype)) return cs;
    for (int i = 0; i < g->np; ++i) {
        const Dims f = g->dims[i][level], c = g->dims[i][level + 1];
        if (dtype == M2S_F64) M2S_TRY(launch_prolong<double>(f, c, (const double*)zc, (double*)z, S(stream)));
        else M2S_TRY(launch_prolong<float>(f, c, (const float*)zc, (float*)z, S(stream)));
    }
    return M2S_OK;
}

m2s_status m2s_mg_vcycle(m2s_grid* g, m2s_dtype dtype, const void* r, void* z, void* stream) {
    M2S_RANGE("m2s_mg_vcycle");
    if (!g || !r || !z || r == z) return M2S_ERR_INVALID_ARG;
    if (is_block(g->op)) return M2S_ERR_INVALID_ARG;
    if (m2s_status cs = check_dtype(g, dtype)) return cs;
    if (dtype == M2S_F64)
        M2S_TRY(vcycle_from<double>(g, (const double*)r, (double*)z, S(stream)));
    else
        M2S_TRY(vcycle_from<float>(g, (const float*)r, (float*)z, S(stream)));
    return M2S_OK;
}

m2s_status m2s_pcg_solve(m2s_grid* g, const double* b, double* x, const m2s_pcg_opts* opts,
                         m2s_pcg_result* out, void* stream) {
    M2S_RANGE("m2s_pcg_solve");
    if (!g || !b || !x || !opts || b == x) return M2S_ERR_INVALID_ARG;
    if (is_block(g->op)) return M2S_ERR_INVALID_ARG;
    m2s_pcg_opts o = *opts;
    if (o.max_iters < 1 || o.max_iters > g->hist_cap || !(o.rtol >= 0)) return M2S_ERR_INVALID_ARG;
    if (o.check_every < 1) o.check_every = 1;
    M2S_TRY(ensure_pcg(g));
    return pcg_batch(g, b, x, o, out, S(stream));
}

m2s_status m2s_kappa_grad(m2s_grid* g, const double* u, const double* lambda, double* dLdkappa,
                          void* stream) {
    M2S_RANGE("m2s_kappa_grad");
    if (!g || !u || !lambda || !dLdkappa || g->op != M2S_OP_DIFF7_KAPPA) return M2S_ERR_INVALID_ARG;
    M2S_TRY(launch_kappa_grad_b(g->batch[0], u, lambda, dLdkappa, S(stream)));
    return M2S_OK;
}

m2s_status m2s_adjoint_solve(m2s_grid* g, const double* u, const double* dLdu, double* lambda,
                             double* dLdkappa, const m2s_pcg_opts* opts, m2s_pcg_result* out,
                             void* stream) {
    M2S_RANGE("m2s_adjoint_solve");
    if (!g || !u || !dLdu || !lambda || !dLdkappa || !opts) return M2S_ERR_INVALID_ARG;
    if (g->op != M2S_OP_DIFF7_KAPPA) return M2S_ERR_INVALID_ARG;
    // A is symmetric (k_f is the same for both cells of a face), so A^T = A
    // and the transposed V-cycle -- transposed sweeps in mirrored order --
    // is the V-cycle itself: the adjoint solve is PCG on A lambda = dL/du.
    m2s_status s = m2s_pcg_solve(g, dLdu, lambda, opts, out, stream);
    if (s != M2S_OK && s != M2S_ERR_NOT_CONVERGED) return s;
    m2s_status s2 = m2s_kappa_grad(g, u, lambda, dLdkappa, stream);
    if (s2 != M2S_OK) return s2;
    M2S_TRY(cudaStreamSynchronize(S(stream)));
    return s;
}

long long m2s_line_penta_work_bytes(int nx, int ny, int nz) {
    if (nx < 1 || ny < 1 || nz < 1) return 0;
    return line_penta_work_doubles(nx, ny, nz) * (long long)sizeof(double);
}

m2s_status m2s_line_penta(int nx, int ny, int nz, int axis, const double* coef, double* rhs,
                          int k, void* work, long long work_bytes, void* stream) {
    M2S_RANGE("m2s_line_penta");
    if (nx < 1 || ny < 1 || nz < 1 || axis < 0 || axis > 2 || k < 1 || k > 8)
        return M2S_ERR_INVALID_ARG;
    if ((i64)nx * ny * nz > (1LL << 34)) return M2S_ERR_INVALID_ARG;
    if (!coef || !rhs || !work || !aligned(coef, 8) || !aligned(rhs, 8) || !aligned(work, 8))
        return M2S_ERR_INVALID_ARG;
    if (work_bytes < m2s_line_penta_work_bytes(nx, ny, nz)) return M2S_ERR_INVALID_ARG;
    const i64 n = (i64)nx * ny * nz;
    // the three arrays must not overlap
    auto disjoint = [](const void* a, i64 na, const void* b, i64 nb) {
        const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
        return x + (uintptr_t)na <= y || y + (uintptr_t)nb <= x;
    };
    const i64 bc = 5 * n * 8, br = (i64)k * n * 8, bw = line_penta_work_doubles(nx, ny, nz) * 8;
    if (!disjoint(coef, bc, rhs, br) || !disjoint(coef, bc, work, bw) || !disjoint(rhs, br, work, bw))
        return M2S_ERR_INVALID_ARG;
    M2S_TRY(launch_line_penta(nx, ny, nz, axis, coef, rhs, k, (double*)work, S(stream)));
    return M2S_OK;
}

m2s_status m2s_ilu0_setup(m2s_grid* g, void* stream) {
    M2S_RANGE("m2s_ilu0_setup");
    if (!g || g->op != M2S_OP_HPCG27) return M2S_ERR_INVALID_ARG;
    cudaStream_t st = S(stream);
    if (!g->ilu_F) M2S_TRY(galloc(g, &g->ilu_F, 27 * g->ltot[0]));
    if (!g->ilu_inv) M2S_TRY(galloc(g, &g->ilu_inv, g->ltot[0]));
    if (!g->ilu_Lw) M2S_TRY(galloc(g, &g->ilu_Lw, 16 * g->ltot[0]));
    if (!g->ilu_Uw) M2S_TRY(galloc(g, &g->ilu_Uw, 16 * g->ltot[0]));
    for (int i = 0; i < g->np; ++i)
        M2S_TRY(launch_ilu_factor(g->dims[i][0], g->ilu_F, g->ilu_inv, st));
    std::vector<Dims> d0(g->np);
    for (int i = 0; i < g->np; ++i) d0[i] = g->dims[i][0];
    M2S_TRY(ilu_wave_setup(d0, g->ltot[0], g->ilu_F, g->ilu_inv, g->ilu_Lw, g->ilu_Uw,
                           &g->ilu_units, st));
    g->last_stream = st;
    return M2S_OK;
}

m2s_status m2s_ilu0_factors(m2s_grid* g, double* out, void* stream) {
    if (!g || g->op != M2S_OP_HPCG27 || !g->ilu_F || !out) return M2S_ERR_INVALID_ARG;
    M2S_TRY(cudaMemcpyAsync(out, g->ilu_F, 27 * g->ltot[0] * sizeof(double),
                            cudaMemcpyDeviceToDevice, S(stream)));
    return M2S_OK;
}

m2s_status m2s_ilu0_apply(m2s_grid* g, const double* r, double* z, void* stream) {
    M2S_RANGE("m2s_ilu0_apply");
    if (!g || g->op != M2S_OP_HPCG27 || !g->ilu_F || !r || !z) return M2S_ERR_INVALID_ARG;
    if (!aligned(r, 8) || !aligned(z, 8)) return M2S_ERR_INVALID_ARG;
    const i64 bytes = g->ltot[0] * 8;
    const uintptr_t a = (uintptr_t)r, b = (uintptr_t)z;
    if (a != b && a < b + (uintptr_t)bytes && b < a + (uintptr_t)bytes) return M2S_ERR_INVALID_ARG;
    cudaStream_t st = S(stream);
    // forward substitution y = L^-1 r into z, then backward z = U^-1 y in
    // place: one wavefront launch each, all problems of the grid
    const int stall = g->ilu_stall_unit;
    g->ilu_stall_unit = -1;
    M2S_TRY(launch_ilu_wave(g->ilu_units, 0, g->spin_ns, g->status, g->ilu_Lw, r, z, stall, st));
    M2S_TRY(launch_ilu_wave(g->ilu_units, 1, g->spin_ns, g->status, g->ilu_Uw, z, z, -1, st));
    g->last_stream = st;
    return M2S_OK;
}

long long m2s_line_btri_work_bytes(int nx, int ny, int nz) {
    if (nx < 1 || ny < 1 || nz < 1) return 0;
    return line_btri_work_doubles(nx, ny, nz) * (long long)sizeof(double);
}

m2s_status m2s_line_btri(int nx, int ny, int nz, int axis, const double* blk, double* rhs,
                         void* work, long long work_bytes, void* stream) {
    M2S_RANGE("m2s_line_btri");
    if (nx < 1 || ny < 1 || nz < 1 || axis < 0 || axis > 2) return M2S_ERR_INVALID_ARG;
    if ((i64)nx * ny * nz > (1LL << 32)) return M2S_ERR_INVALID_ARG;
    if (!blk || !rhs || !work || !aligned(blk, 8) || !aligned(rhs, 8) || !aligned(work, 8))
        return M2S_ERR_INVALID_ARG;
    if (work_bytes < m2s_line_btri_work_bytes(nx, ny, nz)) return M2S_ERR_INVALID_ARG;
    const i64 n = (i64)nx * ny * nz;
    auto disjoint = [](const void* a, i64 na, const void* b, i64 nb) {
        const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
        return x + (uintptr_t)na <= y || y + (uintptr_t)nb <= x;
    };
    const i64 bb = 75 * n * 8, br = 5 * n * 8, bw = line_btri_work_doubles(nx, ny, nz) * 8;
    if (!disjoint(blk, bb, rhs, br) || !disjoint(blk, bb, work, bw) || !disjoint(rhs, br, work, bw))
        return M2S_ERR_INVALID_ARG;
    M2S_TRY(launch_line_btri(nx, ny, nz, axis, blk, rhs, (double*)work, S(stream)));
    return M2S_OK;
}

m2s_status m2s_debug_bounds_read(long long* out) {
    if (!out) return M2S_ERR_INVALID_ARG;
    long long r[3][3];
    M2S_TRY(bounds_read_block(r[0]));
    M2S_TRY(bounds_read_ilu(r[1]));
    M2S_TRY(bounds_read_line(r[2]));
    out[0] = r[0][0] < 0 ? -1 : r[0][0] + r[1][0] + r[2][0];
    out[1] = out[2] = out[3] = -1;
    for (int t = 0; t < 3; ++t)
        if (r[t][0] > 0) {
            out[1] = r[t][1];
            out[2] = r[t][2];
            out[3] = t;
            break;
        }
    return M2S_OK;
}

m2s_status m2s_ssor_sweep(m2s_grid* g, const double* b, double* u, double omega, int n_iters,
                          void* stream) {
    M2S_RANGE("m2s_ssor_sweep");
    if (!g || !b || !u || b == u || !is_block(g->op)) return M2S_ERR_INVALID_ARG;
    if (!(omega > 0.0 && omega < 2.0) || n_iters < 0) return M2S_ERR_INVALID_ARG;
    for (int it = 0; it < n_iters; ++it)
        M2S_TRY(block_ssor_iter(&g->blk, b, u, omega, g->status, g->spin_ns, S(stream)));
    return M2S_OK;
}

}  // extern "C"
