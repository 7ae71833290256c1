// Exact-order 27-point Gauss-Seidel sweeps as a persistent wavefront of
// single-warp units (paper Sec. 4.3.3 SymGS; Sec. 6.1 SewTh: partition,
// crossing dependences, compaction to one monotone counter per producer,
// hyperplane parallelism).  This is the first GPU form of the sweep; the
// allocation-free entry point uses it (it needs no mailbox), the grid
// entry points use the CTA wavefronts of k_wave2.cu (27-point) and
// k_wave7.cu (7-point).  The unit-table helpers below serve all of them.
//
// Every point p is updated in increasing lexicographic order in the sense of
// the method: it sees the NEW values of its lower neighbours and the OLD
// values of its upper neighbours,
//     x_p = (b_p + sum_{q<p} c_pq x_q^new + sum_{q>p} c_pq x_q^old) / a_pp
// (c_pq = -a_pq).  The old part is precomputed as the "old-neighbour sum"
//     Q_p = b_p + sum_{q>p} c_pq x_q^old,
// which is exactly what the previous sweep in the opposite direction leaves
// behind as b_p + (sum of its new lower neighbours): a forward sweep reads Q
// and writes Q' = b + sum_{q<p} c_pq x_q^new for the following backward
// sweep, and vice versa.  A sweep therefore never reads old x.
//
// Backward sweeps are forward sweeps in the reflected index space
// p' = n-1-p (x' = nx-1-x, ...): both stencils are symmetric under the
// reflection, and the reflected lexicographic order is the decreasing order.
//
// Schedule.  The point hyperplane t = x + 2y + 4z satisfies every
// dependence (Eq. "hyperplane" of Sec. 6.1.3 with unit partitions).  Rows
// (y, z) are indexed by (u, v) = (y + z, z); row (u, v) handles x at time
// t - 2u - 2v, and every row it depends on has smaller or equal (u, v), so
// producer/consumer relations between units only point "down-left".
//
// Units.  One warp = one unit: lane i <-> u, register slot j <-> v; the
// first HL lanes and slot 0 are halo rows that REPLAY the producers' rows by
// loading their freshly written values, the other lanes/slots compute.
// Each lane keeps a short window of its rows' newest values in registers;
// neighbour rows come from the lane below (shfl_up) and from the slot below
// (same lane), so within a unit no memory round trip or barrier is needed.
// Units publish their progress (global time completed) in one counter each
// (Thm. 2 of Sec. 6.1.2: one monotone counter per producer suffices); a unit
// waits, with a bounded spin, until its (at most three) producers have
// passed the time it needs.  Units are handed out by an atomic ticket in a
// topological order (v-major, then u), so a waited-for unit has always been
// claimed by a running CTA: no deadlock whatever the residency.  The last
// CTA to leave resets the counters, so consecutive launches need no memset.
#include "m2s_internal.cuh"
#include "m2s_wave_sync.cuh"

#include <algorithm>
#include <climits>
#include <vector>

namespace m2s {

namespace {

using namespace wave;

template <typename T>
struct WaveArgs {
    int nx, ny, nz;
    i64 n, off;
    int rev, publish_every;
    long long spin_ns;
    const T* Qin;
    T* Qout;
    const T* b;
    T* x;
    const int2* origin;
    const int4* prod;
    int n_units;
    int* flags;
    int* ctrl;
    DevStatus* status;
    double* rz;
    int stall_unit;
};

// ---------------------------------------------------------------------------
// 27-point unit: HL = 2 halo lanes, window depth 7.
// ---------------------------------------------------------------------------
template <typename T, int K>
__device__ __forceinline__ void unit27(const WaveArgs<T>& a, int t) {
    constexpr int HL = 2, WD = 7;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int2 org = a.origin[t];
    const int4 pr = a.prod[t];
    const int u = org.x - HL + lane;
    const int tbase = 2 * (org.x - HL) + 2 * (org.y - 1);
    const bool has_prod = pr.x >= 0 || pr.y >= 0 || pr.z >= 0;
    const T inv26 = Lit<T>::inv26();

    bool rv[K];
    i64 base[K];
    const i64 dir = a.rev ? -1 : 1;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int v = org.y - 1 + j;
        const int y = u - v;
        rv[j] = v >= 0 && v < a.nz && y >= 0 && y < a.ny;
        const i64 rb = rv[j] ? ((i64)v * a.ny + y) * a.nx : 0;
        base[j] = a.rev ? a.off + a.n - 1 - rb : a.off + rb;
    }
    T w[K][WD];
#pragma unroll
    for (int j = 0; j < K; ++j)
#pragma unroll
        for (int k = 0; k < WD; ++k) w[j][k] = T(0);

    double rz = 0.0;
    int cached = 0;
    const int S = a.nx + 2 * 31 + 2 * (K - 1);
    const bool halo_lane = lane < HL;
    for (int s = 0; s < S; ++s) {
        const int tnow = s + tbase;
        if (has_prod && tnow + BIAS > cached) {
            if (!wait_producers(a.flags, pr, tnow + BIAS, &cached, a.status, a.spin_ns)) return;
        }
        T up1[K][5], up2[K][3];
#pragma unroll
        for (int j = 0; j < K; ++j) {
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const bool need = (j == 0) ? (k >= 2) : (j == K - 1 ? k < 3 : true);
                up1[j][k] = need ? __shfl_up_sync(FULL, w[j][k], 1) : T(0);
            }
#pragma unroll
            for (int k = 0; k < 3; ++k)
                up2[j][k] = (j < K - 1) ? __shfl_up_sync(FULL, w[j][4 + k], 2) : T(0);
        }
        T nv[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int x = s - 2 * lane - 2 * j;
            const bool in = rv[j] && x >= 0 && x < a.nx;
            nv[j] = T(0);
            if (!in) continue;
            const i64 p = base[j] + dir * x;
            if (j == 0 || halo_lane) {
                nv[j] = __ldcg(a.x + p);
            } else {
                const T N = ((((w[j][0] + up1[j][0]) + (up1[j][1] + up1[j][2])) +
                              ((w[j - 1][0] + w[j - 1][1]) + w[j - 1][2])) +
                             (((up1[j - 1][2] + up1[j - 1][3]) + up1[j - 1][4]) +
                              ((up2[j - 1][0] + up2[j - 1][1]) + up2[j - 1][2])));
                const T q = a.Qin[p];
                const T bp = a.b[p];
                const T xn = (q + N) * inv26;
                a.x[p] = xn;
                if (a.Qout) a.Qout[p] = bp + N;
                if (a.rz) rz = fma((double)bp, (double)xn, rz);
                nv[j] = xn;
            }
        }
#pragma unroll
        for (int j = 0; j < K; ++j) {
#pragma unroll
            for (int k = WD - 1; k > 0; --k) w[j][k] = w[j][k - 1];
            w[j][0] = nv[j];
        }
        if ((s + 1) % a.publish_every == 0) publish(a.flags + t, tnow + BIAS);
    }
    publish(a.flags + t, DONE);
    if (a.rz) {
        for (int o = 16; o > 0; o >>= 1) rz += __shfl_down_sync(FULL, rz, o);
        if (lane == 0) a.rz[t] = rz;
    }
}

template <typename T, int K>
__global__ void __launch_bounds__(32) gs27_wave_kernel(WaveArgs<T> a) {
    run_units(a.n_units, a.flags, a.ctrl, a.status, [&](int t) { unit27<T, K>(a, t); },
              a.stall_unit);
}


}  // namespace

// Unit list of one grid level in ticket (topological) order: units of
// `lanes` computing rows in u and K-1 computing slots in v, u = y + skew*z.
// Producers: the unit to the left (u - lanes), below (v - (K-1)) and, when
// `corner`, below-left.  Empty units (no row inside the grid) are dropped.
// Host only: fills `org` and `prod`.
void build_units_host(int lanes, int skew, int corner, int K, Dims d, std::vector<int2>& org,
                      std::vector<int4>& prod) {
    const int slots = K - 1;
    const int umax = (d.ny - 1) + skew * (d.nz - 1);
    const int NU = umax / lanes + 1;
    const int NV = (d.nz + slots - 1) / slots;
    std::vector<int> index((size_t)NU * NV, -1);
    org.clear();
    for (int V = 0; V < NV; ++V)
        for (int U = 0; U < NU; ++U) {
            const int u0 = U * lanes, v0 = V * slots;
            bool any = false;
            for (int v = v0; v < std::min(v0 + slots, d.nz) && !any; ++v) {
                const int lo = std::max(u0, skew * v);
                const int hi = std::min(u0 + lanes - 1, skew * v + d.ny - 1);
                any = lo <= hi;
            }
            if (!any) continue;
            index[(size_t)V * NU + U] = (int)org.size();
            org.push_back(make_int2(u0, v0));
        }
    prod.assign(org.size(), make_int4(-1, -1, -1, -1));
    for (int V = 0; V < NV; ++V)
        for (int U = 0; U < NU; ++U) {
            const int id = index[(size_t)V * NU + U];
            if (id < 0) continue;
            auto at = [&](int uu, int vv) {
                return (uu < 0 || vv < 0) ? -1 : index[(size_t)vv * NU + uu];
            };
            int4 p;
            p.x = at(U - 1, V);
            p.y = at(U, V - 1);
            p.z = corner ? at(U - 1, V - 1) : -1;
            p.w = -1;
            prod[id] = p;
        }
}

// CTAs of a persistent sweep launch: as many single-warp CTAs as can be
// resident, at most one per unit.
int wave_grid(int n_units, int per_sm) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return std::max(1, std::min(n_units, sms * std::max(1, per_sm)));
}

int wave_blocks_per_sm(int stencil) {
    (void)stencil;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gs27_wave_kernel<double, 5>, 32, 0);
    return std::max(1, per_sm);
}

cudaError_t build_units(int lanes, int skew, int corner, int K, Dims d, int per_sm,
                        WaveUnits* out) {
    std::vector<int2> org;
    std::vector<int4> prod;
    build_units_host(lanes, skew, corner, K, d, org, prod);
    WaveUnits u{};
    u.n_units = (int)org.size();
    u.K = K;
    cudaError_t e = cudaSuccess;
    const size_t nu = std::max<size_t>(org.size(), 1);
    if ((e = cudaMalloc(&u.d_origin, nu * sizeof(int2))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&u.d_prod, nu * sizeof(int4))) != cudaSuccess) { free_wave_units(&u); return e; }
    if ((e = cudaMalloc(&u.d_flags, nu * sizeof(int))) != cudaSuccess) { free_wave_units(&u); return e; }
    if ((e = cudaMalloc(&u.d_ctrl, 2 * sizeof(int))) != cudaSuccess) { free_wave_units(&u); return e; }
    if (!org.empty()) {
        if ((e = cudaMemcpy(u.d_origin, org.data(), org.size() * sizeof(int2),
                            cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemcpy(u.d_prod, prod.data(), prod.size() * sizeof(int4),
                            cudaMemcpyHostToDevice)) != cudaSuccess) {
            free_wave_units(&u);
            return e;
        }
    }
    if ((e = cudaMemset(u.d_flags, 0, nu * sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(u.d_ctrl, 0, 2 * sizeof(int))) != cudaSuccess) {
        free_wave_units(&u);
        return e;
    }
    u.grid = wave_grid(u.n_units, per_sm);
    *out = u;
    return cudaSuccess;
}


void free_wave_units(WaveUnits* u) {
    if (u->d_origin) cudaFree(u->d_origin);
    if (u->d_prod) cudaFree(u->d_prod);
    if (u->d_flags) cudaFree(u->d_flags);
    if (u->d_ctrl) cudaFree(u->d_ctrl);
    if (u->d_mbox) cudaFree(u->d_mbox);
    if (u->d_units) cudaFree(u->d_units);
    if (u->d_dims) cudaFree(u->d_dims);
    if (u->d_rzpre) cudaFree(u->d_rzpre);
    if (u->d_mboff) cudaFree(u->d_mboff);
    *u = WaveUnits{};
}

template <typename T>
static WaveArgs<T> make_args(const WaveUnits& u, const WaveCall& c, Dims d, const T* Qin, T* Qout,
                             const T* b, T* x) {
    WaveArgs<T> a;
    a.nx = d.nx;
    a.ny = d.ny;
    a.nz = d.nz;
    a.n = d.n;
    a.off = d.off;
    a.rev = c.rev;
    a.publish_every = std::max(1, c.publish_every);
    a.spin_ns = c.spin_ns;
    a.Qin = Qin;
    a.Qout = Qout;
    a.b = b;
    a.x = x;
    a.origin = u.d_origin;
    a.prod = u.d_prod;
    a.n_units = u.n_units;
    a.flags = u.d_flags;
    a.ctrl = u.d_ctrl;
    a.status = c.status;
    a.rz = c.rz_partials;
    a.stall_unit = c.stall_unit;
    return a;
}

template <typename T>
cudaError_t launch_gs27_wave(const WaveUnits& u, const WaveCall& c, Dims d, const T* Qin, T* Qout,
                             const T* b, T* x, cudaStream_t st) {
    if (u.n_units == 0) return cudaSuccess;
    WaveArgs<T> a = make_args<T>(u, c, d, Qin, Qout, b, x);
    gs27_wave_kernel<T, 5><<<u.grid, 32, 0, st>>>(a);
    return cudaGetLastError();
}


template cudaError_t launch_gs27_wave<double>(const WaveUnits&, const WaveCall&, Dims,
                                              const double*, double*, const double*, double*,
                                              cudaStream_t);
template cudaError_t launch_gs27_wave<float>(const WaveUnits&, const WaveCall&, Dims, const float*,
                                             float*, const float*, float*, cudaStream_t);

}  // namespace m2s
