// C ABI entry points (include/tmd.h): argument validation, handle management,
// the host-buffer entry points and the velocity-Verlet integrator.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <new>
#include <vector>

#include "tmd_internal.cuh"

namespace tmd {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int g_force_kernel = TMD_FORCE_AUTO;   // tmd_set_force_kernel
int force_kernel() { return g_force_kernel; }

tmd_status cuda_fail(cudaError_t e, const char *what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    (void)cudaGetLastError();   // report a non-sticky error once, not again on the next call
    if (e == cudaErrorMemoryAllocation) return TMD_ERR_OOM;
    return TMD_ERR_CUDA;
}

static bool g_graphs = true;   // tmd_set_graphs
static int64_t g_replays = 0;  // graph launches that replayed a captured sequence

// Run launch() (a fixed sequence of launches on s) through gc: eagerly the
// first time a key is seen, captured into a graph the second time, replayed
// after that.  Eager whenever graphs are off, profiling is on (per-launch
// events) or s is the legacy default stream (which cannot be captured).
template <typename F>
tmd_status graphed(GraphCache &gc, const std::vector<uintptr_t> &key, cudaStream_t s, F &&launch) {
    if (!g_graphs || s == nullptr || profiling_on()) return launch();
    if (gc.exec && gc.key == key) {
        TMD_CUDA(cudaGraphLaunch(gc.exec, s));
        add_launches(gc.kernels);
        ++g_replays;
        return TMD_OK;
    }
    if (gc.pending != key) {
        gc.pending = key;
        return launch();
    }
    cudaGraph_t g = nullptr;
    TMD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const tmd_status st = launch();
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st != TMD_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
    int64_t nk = 0;
    for (cudaGraphNode_t v : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(v, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++nk;
    }
    if (gc.exec) {
        cudaGraphExecDestroy(gc.exec);
        gc.exec = nullptr;
    }
    const cudaError_t ei = cudaGraphInstantiate(&gc.exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        gc.exec = nullptr;
        return cuda_fail(ei, "cudaGraphInstantiate");
    }
    gc.key = key;
    gc.kernels = nk;
    TMD_CUDA(cudaGraphLaunch(gc.exec, s));   // the capture itself counted these launches
    return TMD_OK;
}

// addresses and sizes a neighbour table's evaluation launches depend on
void nlist_key(const tmd_nlist &nl, std::vector<uintptr_t> &k) {
    const void *p[] = {nl.perm, nl.beg, nl.end, nl.nbr, nl.shift, nl.G, nl.dG, nl.P, nl.Fq, nl.part,
                       nl.ph, nl.pl, nl.pq, nl.pq2, nl.npair, nl.sp};
    for (const void *q : p) k.push_back((uintptr_t)q);
    k.push_back((uintptr_t)nl.n_active);
}

void model_key(const tmd_model *m, std::vector<uintptr_t> &k) {
    k.push_back((uintptr_t)m);
    k.push_back((uintptr_t)m->dm.precision);
    k.push_back((uintptr_t)m->dm.tile_rows);
    k.push_back((uintptr_t)m->dm.pair_bps);
    k.push_back((uintptr_t)m->dm.rtab);
    k.push_back((uintptr_t)m->dm.rtab_n);
    k.push_back((uintptr_t)m->dm.rtab_scale);
    k.push_back((uintptr_t)tmd::network_kernel());
    k.push_back((uintptr_t)tmd::force_kernel());
}

uintptr_t bits_of(double x) {
    uintptr_t u = 0;
    std::memcpy(&u, &x, sizeof(double) < sizeof(uintptr_t) ? sizeof(double) : sizeof(uintptr_t));
    return u;
}

namespace {

// eV/(A amu) -> A/fs^2
constexpr double ACC_CONV = 1.0 / 103.6427;
constexpr double FQ_UNIT = 1.0 / 4294967296.0;   // the force accumulator's unit, 2^-32 eV/A
constexpr double KB_EV = 8.617333262e-5;

// Half kick and drift.  Positions are not wrapped here: the neighbour table's
// image shifts refer to the positions at the last build, so atoms move
// continuously until the next rebuild, which wraps them first.
// First half kick and drift; the drifted positions are also written as the
// pair kernels' hi/lo split (ph, pl), so that the evaluation that follows
// need not form it again.
__global__ void k_vv_first(double *__restrict__ pos, double *__restrict__ vel, const float *__restrict__ F,
                           const double *__restrict__ inv_mass, int64_t n, double dt,
                           const double *__restrict__ pos_ref, double lim2, int32_t *__restrict__ flag,
                           float4 *__restrict__ ph, float4 *__restrict__ pl) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double h = 0.5 * dt * inv_mass[i] * ACC_CONV;
    double d2 = 0.0;
    float sh[3], sl[3];
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        const double v = vel[3 * i + x] + h * (double)F[3 * i + x];
        const double p = pos[3 * i + x] + dt * v;
        vel[3 * i + x] = v;
        pos[3 * i + x] = p;
        grid_split(p, sh[x], sl[x]);
        const double d = p - pos_ref[3 * i + x];
        d2 += d * d;
    }
    if (ph) {
        ph[i] = make_float4(sh[0], sh[1], sh[2], 0.f);
        pl[i] = make_float4(sl[0], sl[1], sl[2], 0.f);
    }
    // bit 0: moved more than skin/2 (rebuild); bit 1: more than 0.7 skin/2
    // (close to it: the step loop stops running steps ahead, see tmd_step)
    if (d2 > 0.49 * lim2) atomicOr(flag, d2 > lim2 ? 3 : 2);
}

// Wrap positions into [0, L) on periodic axes (before a neighbour rebuild).
// Wrap positions into [0, L) on periodic axes (before a neighbour rebuild);
// a wrapped atom's hi/lo split (ph, pl) is formed again.
__global__ void k_wrap(double *__restrict__ pos, int64_t n, double L0, double L1, double L2, int p0, int p1,
                       int p2, float4 *__restrict__ ph, float4 *__restrict__ pl) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double L[3] = {L0, L1, L2};
    const int pb[3] = {p0, p1, p2};
    bool moved = false;
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        if (!pb[x]) continue;
        double p = pos[3 * i + x];
        if (p < 0.0 || p >= L[x]) {  // rare: only atoms that left the box
            p = p - floor(p * (1.0 / L[x])) * L[x];
            if (p >= L[x]) p -= L[x];
            if (p < 0.0) p += L[x];
            pos[3 * i + x] = p;
            moved = true;
        }
    }
    if (moved && ph) {
        float sh[3], sl[3];
#pragma unroll
        for (int x = 0; x < 3; ++x) grid_split(pos[3 * i + x], sh[x], sl[x]);
        ph[i] = make_float4(sh[0], sh[1], sh[2], 0.f);
        pl[i] = make_float4(sl[0], sl[1], sl[2], 0.f);
    }
}

// the second half kick fused with the conversion of the pair passes' force
// accumulator (int64, 2^-32 eV/A) to the FP32 forces it also writes: the
// same values as the conversion and the kick launched one after the other
__global__ void k_vv_second_fq(double *__restrict__ vel, const long long *__restrict__ Fq, float *__restrict__ F,
                               const double *__restrict__ inv_mass, int64_t n, double dt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double h = 0.5 * dt * inv_mass[i] * ACC_CONV;
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        const float f = (float)((double)Fq[3 * i + x] * FQ_UNIT);
        F[3 * i + x] = f;
        vel[3 * i + x] += h * (double)f;
    }
}

// block partials of sum m v_a v_b (FP64), 6 components
__global__ void k_kinetic(const double *__restrict__ vel, const double *__restrict__ mass, int64_t n,
                          double *__restrict__ part) {
    __shared__ double s[6][8];
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double m = mass[i], x = vel[3 * i], y = vel[3 * i + 1], z = vel[3 * i + 2];
        v[0] += m * x * x; v[1] += m * y * y; v[2] += m * z * z;
        v[3] += m * x * y; v[4] += m * x * z; v[5] += m * y * z;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < 6; ++t) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[t] += __shfl_xor_sync(0xffffffffu, v[t], o);
        if (lane == 0) s[t][warp] = v[t];
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double acc = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) acc += s[threadIdx.x][w];
        part[(size_t)blockIdx.x * 6 + threadIdx.x] = acc;
    }
}

__global__ void k_kinetic_total(const double *__restrict__ part, int nb, double *__restrict__ out) {
    if (threadIdx.x < 6) {
        double acc = 0.0;
        for (int b = 0; b < nb; ++b) acc += part[(size_t)b * 6 + threadIdx.x];
        out[threadIdx.x] = acc;
    }
}

__global__ void k_inv_mass(const double *__restrict__ mass, double *__restrict__ inv, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) inv[i] = 1.0 / mass[i];
}

// velocity-Verlet halves and wrap for the atoms of the active systems of a
// batch.  The first half kick and drift also run each system's skin check:
// an atom that moved more than skin/2 since its system's last table build
// sets moved[system] (lim2 = (skin/2)^2; no check when moved is null).
__global__ void k_vv_first_b(double *__restrict__ pos, double *__restrict__ vel, const float *__restrict__ F,
                             const double *__restrict__ inv_mass, int64_t n, double dt,
                             const int32_t *__restrict__ sys_of, const uint8_t *__restrict__ active,
                             const double *__restrict__ pos_ref, double lim2, int32_t *__restrict__ moved) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int sys = sys_of[i];
    if (!active[sys]) return;
    const double h = 0.5 * dt * inv_mass[i] * ACC_CONV;
    double d2 = 0.0;
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        const double v = vel[3 * i + x] + h * (double)F[3 * i + x];
        const double p = pos[3 * i + x] + dt * v;
        vel[3 * i + x] = v;
        pos[3 * i + x] = p;
        if (moved) {
            const double d = p - pos_ref[3 * i + x];
            d2 += d * d;
        }
    }
    if (moved && d2 > lim2) atomicOr(&moved[sys], 1);
}

// pos_ref = pos for the atoms of the flagged systems (after their rebuild)
__global__ void k_copy_ref_b(const double *__restrict__ pos, double *__restrict__ pos_ref, int64_t n,
                             const int32_t *__restrict__ sys_of, const uint8_t *__restrict__ flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flag[sys_of[i]]) return;
#pragma unroll
    for (int x = 0; x < 3; ++x) pos_ref[3 * i + x] = pos[3 * i + x];
}

// The evaluation order of the active atoms: grouped by species, within a
// species by system (in the order of the active list) and atom index.
// rank[i] = the index of atom i among the atoms of its species in its system;
// pbase[sys * MAX_SPECIES + t] = the first perm position of that block.
__global__ void k_eval_perm(int64_t n, const int32_t *__restrict__ sys_of, const uint8_t *__restrict__ active,
                            const int32_t *__restrict__ types, const int32_t *__restrict__ rank,
                            const int64_t *__restrict__ pbase, int32_t *__restrict__ perm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int sys = sys_of[i];
    if (!active[sys]) return;
    perm[pbase[(int64_t)sys * TMD_MAX_SPECIES + types[i]] + rank[i]] = (int32_t)i;
}

// Move the segments of a fresh build (scratch table, the atoms in sperm) into
// the resident table: each system's entries go to its own region of the pool
// (region[2 sys] = first entry, region[2 sys + 1] = capacity), reserved per
// atom from fill[sys].  A region too small for its system's entries gets
// empty segments and overflow = 1; fill then holds the entries it needed.
// One warp per atom.
__global__ void k_region_copy(const int64_t *__restrict__ sbeg, const int64_t *__restrict__ send,
                              const int32_t *__restrict__ snbr, const char4 *__restrict__ sshift,
                              const int32_t *__restrict__ sperm, int64_t nr, const int32_t *__restrict__ sys_of,
                              const int64_t *__restrict__ region, unsigned long long *__restrict__ fill,
                              int64_t *__restrict__ beg, int64_t *__restrict__ end, int32_t *__restrict__ nbr,
                              char4 *__restrict__ shift, int32_t *__restrict__ overflow) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < nr; p += nw) {
        const int i = sperm[p];
        const int sys = sys_of[i];
        const int64_t b0 = sbeg[i], len = send[i] - b0;
        unsigned long long off = 0;
        if (lane == 0) off = atomicAdd(&fill[sys], (unsigned long long)len);
        off = __shfl_sync(0xffffffffu, off, 0);
        const int64_t base = region[2 * sys], cap = region[2 * sys + 1];
        if ((int64_t)off + len > cap) {
            if (lane == 0) {
                beg[i] = end[i] = base;
                atomicOr(overflow, 1);
            }
            continue;
        }
        const int64_t d0 = base + (int64_t)off;
        for (int64_t c = lane; c < len; c += 32) {
            nbr[d0 + c] = snbr[b0 + c];
            shift[d0 + c] = sshift[b0 + c];
        }
        if (lane == 0) {
            beg[i] = d0;
            end[i] = d0 + len;
        }
    }
}

__global__ void k_vv_second_b(double *__restrict__ vel, const float *__restrict__ F, const double *__restrict__ inv_mass,
                              int64_t n, double dt, const int32_t *__restrict__ sys_of,
                              const uint8_t *__restrict__ active) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !active[sys_of[i]]) return;
    const double h = 0.5 * dt * inv_mass[i] * ACC_CONV;
#pragma unroll
    for (int x = 0; x < 3; ++x) vel[3 * i + x] += h * (double)F[3 * i + x];
}

__global__ void k_wrap_b(double *__restrict__ pos, int64_t n, const SysParams *__restrict__ sp,
                         const int32_t *__restrict__ sys_of, const uint8_t *__restrict__ active) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int sys = sys_of[i];
    if (!active[sys]) return;
    const SysParams &q = sp[sys];
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        if (!q.pbc[x]) continue;
        double p = pos[3 * i + x];
        if (p < 0.0 || p >= q.L[x]) {
            p = p - floor(p * (1.0 / q.L[x])) * q.L[x];
            if (p >= q.L[x]) p -= q.L[x];
            if (p < 0.0) p += q.L[x];
            pos[3 * i + x] = p;
        }
    }
}

bool finite_all(const double *p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

inline uint16_t to_bf16(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);
    const uint32_t rounding = 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)((u + rounding) >> 16);
}

tmd_status check_box(const double box[3], const int32_t pbc[3]) {
    if (!box || !pbc) {
        set_error("box and pbc must be non-NULL host arrays");
        return TMD_ERR_INVALID_ARG;
    }
    for (int x = 0; x < 3; ++x)
        if (!(std::isfinite(box[x]) && box[x] > 0.0)) {
            set_error("box[%d] = %g must be finite and > 0", x, box[x]);
            return TMD_ERR_INVALID_ARG;
        }
    return TMD_OK;
}

}  // namespace
}  // namespace tmd

using namespace tmd;

extern "C" {

const char *tmd_status_string(int status) {
    switch (status) {
        case TMD_OK: return "TMD_OK";
        case TMD_ERR_INVALID_ARG: return "TMD_ERR_INVALID_ARG";
        case TMD_ERR_CAPACITY: return "TMD_ERR_CAPACITY";
        case TMD_ERR_CUDA: return "TMD_ERR_CUDA";
        case TMD_ERR_OOM: return "TMD_ERR_OOM";
        case TMD_ERR_TIMEOUT: return "TMD_ERR_TIMEOUT";
        case TMD_ERR_UNIMPLEMENTED: return "TMD_ERR_UNIMPLEMENTED";
        default: return "TMD_ERR_UNKNOWN";
    }
}

const char *tmd_last_error(void) { return g_err; }

const char *tmd_version(void) { return "tensormd-gb300 0.1 (sm_103a)"; }

// --------------------------------------------------------------------- model
tmd_status tmd_model_create(const tmd_model_desc *d, tmd_model **out) {
    g_err[0] = 0;
    if (!d || !out) { set_error("null descriptor or output"); return TMD_ERR_INVALID_ARG; }
    *out = nullptr;
    const int S = d->n_species, K = d->n_radial, L = d->n_hidden;
    if (S < 1 || S > TMD_MAX_SPECIES) { set_error("n_species %d outside [1, %d]", S, TMD_MAX_SPECIES); return TMD_ERR_INVALID_ARG; }
    if (K != 8 && K != 16 && K != 32 && K != 64 && K != 128) {
        set_error("n_radial %d: the library supports 8, 16, 32, 64, 128", K);
        return TMD_ERR_UNIMPLEMENTED;
    }
    // species counts with kernel instances (network inputs S K 4 up to 640)
    const int s_max = K <= 32 ? 5 : (K == 64 ? 2 : 1);
    if (S > s_max) { set_error("n_radial %d supports at most %d species", K, s_max); return TMD_ERR_UNIMPLEMENTED; }
    if (!(std::isfinite(d->rc) && d->rc > 0.0)) { set_error("rc must be finite and > 0"); return TMD_ERR_INVALID_ARG; }
    if (L < 1 || L > TMD_MAX_HIDDEN) { set_error("n_hidden %d outside [1, %d]", L, TMD_MAX_HIDDEN); return TMD_ERR_INVALID_ARG; }
    if (!d->widths || !d->weights || !d->mu || !d->eta) { set_error("null widths/weights/mu/eta"); return TMD_ERR_INVALID_ARG; }
    if (d->activation != TMD_ACT_TANH && d->activation != TMD_ACT_SQUAREPLUS) { set_error("unknown activation"); return TMD_ERR_INVALID_ARG; }
    if (d->activation == TMD_ACT_SQUAREPLUS && !(d->squareplus_b > 0.0)) { set_error("squareplus_b must be > 0"); return TMD_ERR_INVALID_ARG; }
    if (d->precision != TMD_PREC_FP32 && d->precision != TMD_PREC_BF16) { set_error("unknown precision"); return TMD_ERR_INVALID_ARG; }
    const int Dd = S * K * 4;
    int dims[MAX_LAYERS + 1];
    dims[0] = Dd;
    for (int l = 0; l < L; ++l) {
        const int w = d->widths[l];
        if (w < 4 || w > TMD_MAX_WIDTH || w % 4) { set_error("width %d must be a multiple of 4 in [4, %d]", w, TMD_MAX_WIDTH); return TMD_ERR_INVALID_ARG; }
        dims[l + 1] = w;
    }
    dims[L + 1] = 1;
    if (!finite_all(d->mu, (size_t)S * S * K) || !finite_all(d->eta, (size_t)S * S * K)) { set_error("non-finite mu/eta"); return TMD_ERR_INVALID_ARG; }
    for (size_t i = 0; i < (size_t)S * S * K; ++i)
        if (!(d->eta[i] >= 0.0)) { set_error("eta must be >= 0"); return TMD_ERR_INVALID_ARG; }
    // per-species float counts
    size_t nf = 0, nb = 0;
    int off_f[MAX_LAYERS], off_b[MAX_LAYERS];
    for (int l = 0; l <= L; ++l) {
        off_f[l] = (int)nf;
        off_b[l] = (int)nb;
        nf += (size_t)dims[l] * dims[l + 1] + dims[l + 1];
        nb += (size_t)dims[l] * dims[l + 1];
    }
    size_t nflat = 0;
    for (int l = 0; l <= L; ++l) nflat += (size_t)dims[l] * dims[l + 1] + dims[l + 1];
    for (int s = 0; s < S; ++s) {
        if (!d->weights[s]) { set_error("weights[%d] is NULL", s); return TMD_ERR_INVALID_ARG; }
        if (!finite_all(d->weights[s], nflat)) { set_error("non-finite weight in species %d", s); return TMD_ERR_INVALID_ARG; }
    }
    // host staging: radial | per species fwd fp32 | bwd fp32 | fwd bf16 | bwd bf16  (16 B aligned parts)
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t b_rad = al(sizeof(float4) * S * S * K);
    const size_t b_f = al(sizeof(float) * nf), b_b = al(sizeof(float) * nb);
    const size_t b_hf = al(sizeof(uint16_t) * nf), b_hb = al(sizeof(uint16_t) * nb);
    const size_t total = b_rad + S * (b_f + b_b + b_hf + b_hb);
    std::vector<unsigned char> host(total, 0);
    float4 *rad = reinterpret_cast<float4 *>(host.data());
    const double log2e = 1.4426950408889634;
    for (int i = 0; i < S * S * K; ++i) {
        const float mu_hi = (float)d->mu[i];
        const float mu_lo = (float)(d->mu[i] - (double)mu_hi);
        rad[i] = make_float4(mu_hi, mu_lo, (float)(d->eta[i] * log2e), (float)(2.0 * d->eta[i]));
    }
    tmd_model *m = new (std::nothrow) tmd_model();
    if (!m) { set_error("host allocation failed"); return TMD_ERR_OOM; }
    cudaError_t e = cudaMalloc(&m->dev_block, total);
    if (e != cudaSuccess) { delete m; cudaGetLastError(); set_error("cudaMalloc model: %s", cudaGetErrorString(e)); return TMD_ERR_OOM; }
    m->dev_bytes = total;
    DevModel &dm = m->dm;
    std::memset(&dm, 0, sizeof(dm));
    dm.S = S; dm.K = K; dm.L = L; dm.act = d->activation; dm.Dd = Dd; dm.nlayers = L + 1;
    dm.precision = d->precision;
    dm.rc = (float)d->rc; dm.rc2 = (float)(d->rc * d->rc); dm.inv_rc = (float)(1.0 / d->rc);
    dm.rc2h = (float)(d->rc * d->rc);
    dm.rc2l = (float)(d->rc * d->rc - (double)dm.rc2h);
    dm.sp_b = (float)d->squareplus_b;
    for (int l = 0; l <= L + 1; ++l) dm.dims[l] = dims[l];
    for (int l = 0; l <= L; ++l) { dm.off_f[l] = off_f[l]; dm.off_b[l] = off_b[l]; }
    unsigned char *dev = static_cast<unsigned char *>(m->dev_block);
    dm.radial = reinterpret_cast<const float4 *>(dev);
    size_t cur = b_rad;
    for (int s = 0; s < S; ++s) {
        float *hf = reinterpret_cast<float *>(host.data() + cur);
        float *hbk = reinterpret_cast<float *>(host.data() + cur + b_f);
        uint16_t *qf = reinterpret_cast<uint16_t *>(host.data() + cur + b_f + b_b);
        uint16_t *qb = reinterpret_cast<uint16_t *>(host.data() + cur + b_f + b_b + b_hf);
        const double *w = d->weights[s];
        size_t o = 0;
        for (int l = 0; l <= L; ++l) {
            const int in = dims[l], outd = dims[l + 1];
            for (int r = 0; r < outd; ++r)
                for (int c = 0; c < in; ++c) {
                    const float v = (float)w[o + (size_t)r * in + c];
                    hf[off_f[l] + (size_t)c * outd + r] = v;      // W^T [in][out]
                    hbk[off_b[l] + (size_t)r * in + c] = v;       // W [out][in]
                    qf[off_f[l] + (size_t)c * outd + r] = to_bf16(v);
                    qb[off_b[l] + (size_t)r * in + c] = to_bf16(v);
                }
            o += (size_t)in * outd;
            for (int r = 0; r < outd; ++r) hf[off_f[l] + (size_t)in * outd + r] = (float)w[o + r];
            o += outd;
        }
        dm.wf[s] = reinterpret_cast<const float *>(dev + cur);
        dm.wb[s] = reinterpret_cast<const float *>(dev + cur + b_f);
        dm.hf[s] = reinterpret_cast<const uint16_t *>(dev + cur + b_f + b_b);
        dm.hb[s] = reinterpret_cast<const uint16_t *>(dev + cur + b_f + b_b + b_hf);
        cur += b_f + b_b + b_hf + b_hb;
    }
    e = cudaMemcpy(m->dev_block, host.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(m->dev_block); delete m; return cuda_fail(e, "cudaMemcpy model"); }
    m->precision = d->precision;
    m->mu.assign(d->mu, d->mu + (size_t)S * S * K);
    m->eta.assign(d->eta, d->eta + (size_t)S * S * K);
    m->rc_exact = d->rc;
    {
        const tmd_status su = tmd::mlp_umma_build(m, d->weights);
        if (su != TMD_OK) { cudaFree(m->dev_block); delete m; return su; }
    }
    if (tmd::mlp_smem_tr_public(m->dm, 32) > 227 * 1024) {
        set_error("network too wide: the activations of a 32-atom tile exceed the shared memory of an SM");
        cudaFree(m->dev_block);
        if (m->dev_umma) cudaFree(m->dev_umma);
        delete m;
        return TMD_ERR_UNIMPLEMENTED;
    }
    if (d->precision == TMD_PREC_BF16) {
        tmd_status st = tmd_model_set_precision(m, TMD_PREC_BF16);
        if (st != TMD_OK) { cudaFree(m->dev_block); if (m->dev_umma) cudaFree(m->dev_umma); delete m; return st; }
    }
    *out = m;
    return TMD_OK;
}

tmd_status tmd_model_destroy(tmd_model *m) {
    if (!m) return TMD_OK;
    if (m->dev_block) cudaFree(m->dev_block);
    if (m->dev_rtab) cudaFree(m->dev_rtab);
    if (m->dev_umma) cudaFree(m->dev_umma);
    delete m;
    return TMD_OK;
}

extern "C++" {
namespace {

bool table_ppa_ok(int32_t ppa) { return ppa >= 16 && ppa <= 1024 && (ppa & (ppa - 1)) == 0; }

void table_clear(tmd_model *m) {
    if (m->dev_rtab) {
        cudaFree(m->dev_rtab);
        m->dev_rtab = nullptr;
    }
    m->dm.rtab = nullptr;
    m->dm.rtab_scale = 0.f;
    m->dm.rtab_n = 0;
}

// Build and upload the tabulated radial basis from node values:
// node(p, k, g, H, dH) gives H and H' of species pair p, channel k at
// r_g = g / ppa (only called for r_g < rc; nodes from rc on are zero, the
// cutoff folded into the table).  Interval g = [g h, (g + 1) h), h = 1/ppa,
// holds the cubic Hermite polynomial through H and H' at both ends as
// coefficients in t = (r - g h)/h: H = c0 + c1 t + c2 t^2 + c3 t^3,
// H' = (c1 + 2 c2 t + 3 c3 t^2) ppa.  The coefficients are formed in FP64 and
// rounded to FP32 (storing node values instead would lose H' to cancellation
// in (H_g+1 - H_g) ppa once the grid is fine).  Intervals up to
// floor(rc ppa) + 1: an FP32 r just below rc can round into the interval one
// past floor(rc ppa) when rc ppa sits within an ulp of an integer.
template <typename Node>
tmd_status table_build(tmd_model *m, int32_t ppa, Node &&node) {
    const int S = m->dm.S, K = m->dm.K;
    const double rcd = m->rc_exact;
    const int n = (int)std::floor(rcd * ppa) + 2;
    std::vector<float> h((size_t)S * S * n * 4 * K, 0.f);
    const double hs = 1.0 / ppa;
    auto at = [&](int p, int k, int g, double &H, double &dH) {
        H = dH = 0.0;
        if ((double)g * hs < rcd) node(p, k, g, H, dH);
    };
    for (int p = 0; p < S * S; ++p)
        for (int g = 0; g < n; ++g)
            for (int k = 0; k < K; ++k) {
                double y0, d0, y1, d1;
                at(p, k, g, y0, d0);
                at(p, k, g + 1, y1, d1);
                const double dy = y1 - y0, s0 = d0 * hs, s1 = d1 * hs;
                float *c = &h[(((size_t)p * n + g) * K + k) * 4];
                c[0] = (float)y0;
                c[1] = (float)s0;
                c[2] = (float)(3.0 * dy - 2.0 * s0 - s1);
                c[3] = (float)(-2.0 * dy + s0 + s1);
            }
    cudaError_t e = cudaMalloc(&m->dev_rtab, sizeof(float) * h.size());
    if (e != cudaSuccess) { m->dev_rtab = nullptr; return cuda_fail(e, "cudaMalloc radial table"); }
    e = cudaMemcpy(m->dev_rtab, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(m->dev_rtab); m->dev_rtab = nullptr; return cuda_fail(e, "cudaMemcpy radial table"); }
    m->dm.rtab = m->dev_rtab;
    m->dm.rtab_scale = (float)ppa;
    m->dm.rtab_n = n;
    return TMD_OK;
}

}  // namespace
}  // extern "C++"

tmd_status tmd_model_set_radial_table(tmd_model *m, int32_t ppa) {
    g_err[0] = 0;
    if (!m || ppa < 0 || (ppa != 0 && !table_ppa_ok(ppa))) {
        set_error("points_per_angstrom must be 0 or a power of two in [16, 1024]");
        return TMD_ERR_INVALID_ARG;
    }
    table_clear(m);
    if (ppa == 0) return TMD_OK;
    // H_k = f_k f_c and H'_k of the model's Gaussians at the grid points, FP64
    const int K = m->dm.K;
    const double rcd = m->rc_exact, pi = 3.14159265358979323846, hs = 1.0 / ppa;
    return table_build(m, ppa, [&](int p, int k, int g, double &H, double &dH) {
        const double r = g * hs;
        const double fc = 0.5 * (std::cos(pi * r / rcd) + 1.0);
        const double dfc = -0.5 * pi / rcd * std::sin(pi * r / rcd);
        const double mu = m->mu[(size_t)p * K + k], eta = m->eta[(size_t)p * K + k];
        const double t = r - mu, f = std::exp(-eta * t * t);
        H = f * fc;
        dH = f * (-2.0 * eta * t * fc + dfc);
    });
}

tmd_status tmd_model_set_radial_table_values(tmd_model *m, int32_t ppa, int32_t n_points, const double *H,
                                             const double *dH) {
    g_err[0] = 0;
    if (!m || !table_ppa_ok(ppa) || !H || !dH) {
        set_error("points_per_angstrom must be a power of two in [16, 1024]; H and dH non-NULL");
        return TMD_ERR_INVALID_ARG;
    }
    const int S = m->dm.S, K = m->dm.K;
    const int need = (int)std::ceil(m->rc_exact * ppa);   // every grid point below rc
    if (n_points < need || n_points > need + 4096) {
        set_error("n_points %d: the grid must cover [0, rc): at least %d points per species pair", n_points, need);
        return TMD_ERR_INVALID_ARG;
    }
    const size_t total = (size_t)S * S * n_points * K;
    if (!finite_all(H, total) || !finite_all(dH, total)) {
        set_error("non-finite table value");
        return TMD_ERR_INVALID_ARG;
    }
    table_clear(m);
    // caller's values at r_g = g / ppa, [S][S][n_points][K]
    return table_build(m, ppa, [&](int p, int k, int g, double &h, double &d) {
        const size_t i = ((size_t)p * n_points + g) * K + k;
        h = H[i];
        d = dH[i];
    });
}

tmd_status tmd_model_set_precision(tmd_model *m, int32_t precision) {
    if (!m || (precision != TMD_PREC_FP32 && precision != TMD_PREC_BF16)) {
        set_error("bad model or precision");
        return TMD_ERR_INVALID_ARG;
    }
    if (precision == TMD_PREC_BF16)
        for (int l = 0; l <= m->dm.L; ++l)
            if (m->dm.dims[l] % 16) {
                set_error("the BF16 network needs layer widths that are multiples of 16 (layer %d has %d)", l,
                          m->dm.dims[l]);
                return TMD_ERR_UNIMPLEMENTED;
            }
    if (precision == TMD_PREC_BF16 && !tmd::mlp_umma_supported(m->dm) && tmd::mlp_bf16_smem_bytes(m->dm) > 227 * 1024) {
        set_error("network too wide for the BF16 tile (64 atoms) in the shared memory of an SM");
        return TMD_ERR_UNIMPLEMENTED;
    }
    m->precision = precision;
    m->dm.precision = precision;
    return TMD_OK;
}

tmd_status tmd_set_network_kernel(int32_t kind) {
    g_err[0] = 0;
    if (kind < TMD_NET_AUTO || kind > TMD_NET_MMA_SYNC) {
        set_error("network kernel must be TMD_NET_AUTO, TMD_NET_TCGEN05 or TMD_NET_MMA_SYNC");
        return TMD_ERR_INVALID_ARG;
    }
    tmd::g_network_kernel = kind;
    return TMD_OK;
}

tmd_status tmd_set_force_kernel(int32_t kind) {
    g_err[0] = 0;
    if (kind < TMD_FORCE_AUTO || kind > TMD_FORCE_TENSOR) {
        set_error("force kernel must be TMD_FORCE_AUTO, TMD_FORCE_SIMT or TMD_FORCE_TENSOR");
        return TMD_ERR_INVALID_ARG;
    }
    tmd::g_force_kernel = kind;
    return TMD_OK;
}

tmd_status tmd_device_status(int32_t *bits) {
    g_err[0] = 0;
    if (!bits) { set_error("null output"); return TMD_ERR_INVALID_ARG; }
    tmd_status st = tmd::umma_status(bits);
    if (st != TMD_OK) return st;
    if (*bits & tmd::DEV_ERR_TIMEOUT) {
        set_error("a bounded wait of a tensor-core kernel gave up; the results since the last check are invalid");
        return TMD_ERR_TIMEOUT;
    }
    return TMD_OK;
}

tmd_status tmd_selftest_bounded_wait(int32_t *gave_up) {
    g_err[0] = 0;
    if (!gave_up) { set_error("null output"); return TMD_ERR_INVALID_ARG; }
    return tmd::wait_probe(gave_up);
}

tmd_status tmd_set_graphs(int32_t on) {
    g_graphs = on != 0;
    return TMD_OK;
}

int64_t tmd_graph_replays(void) { return g_replays; }

tmd_status tmd_model_set_tuning(tmd_model *m, const tmd_tuning *t) {
    g_err[0] = 0;
    if (!m || !t || (t->tile_rows != 0 && t->tile_rows != 32 && t->tile_rows != 64 && t->tile_rows != 128) ||
        t->pair_blocks_per_sm < 0 || t->pair_blocks_per_sm > 64) {
        set_error("bad model or tuning (tile_rows 0/32/64/128, pair_blocks_per_sm 0..64)");
        return TMD_ERR_INVALID_ARG;
    }
    m->dm.tile_rows = t->tile_rows;
    m->dm.pair_bps = t->pair_blocks_per_sm;
    return TMD_OK;
}

tmd_status tmd_model_get_tuning(const tmd_model *m, tmd_tuning *t) {
    if (!m || !t) { set_error("null model or output"); return TMD_ERR_INVALID_ARG; }
    t->tile_rows = m->dm.tile_rows;
    t->pair_blocks_per_sm = m->dm.pair_bps;
    t->ms = 0.f;
    return TMD_OK;
}

}  // extern "C"

namespace {

// Time run() (one evaluation enqueued on s) for every candidate tile shape and
// keep the fastest in the model: one untimed run per candidate (it also sizes
// the workspaces), then three timed back to back.
template <typename F>
tmd_status tune_shapes(tmd_model *m, cudaStream_t s, tmd_tuning *best, F &&run) {
    const int rows_fp32[3] = {32, 64, 128};
    const int bps[4] = {4, 8, 16, 32};
    const int nrows = (m->dm.precision == TMD_PREC_FP32) ? 3 : 1;
    cudaEvent_t e0, e1;
    TMD_CUDA(cudaEventCreate(&e0));
    TMD_CUDA(cudaEventCreate(&e1));
    tmd_tuning top = {0, 0, 1e30f};
    const tmd::DevModel keep = m->dm;
    tmd_status st = TMD_OK;
    for (int r = 0; r < nrows && st == TMD_OK; ++r) {
        m->dm.tile_rows = (m->dm.precision == TMD_PREC_FP32) ? rows_fp32[r] : 0;
        if (m->dm.tile_rows && !tmd::mlp_rows_ok(m->dm, m->dm.tile_rows)) continue;
        for (int b = 0; b < 4 && st == TMD_OK; ++b) {
            m->dm.pair_bps = bps[b];
            if ((st = run()) != TMD_OK) break;
            if (cudaEventRecord(e0, s) != cudaSuccess) { st = TMD_ERR_CUDA; break; }
            for (int k = 0; k < 3 && st == TMD_OK; ++k) st = run();
            if (st != TMD_OK) break;
            if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) { st = TMD_ERR_CUDA; break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= 3.f;
            if (ms < top.ms) top = {m->dm.tile_rows, m->dm.pair_bps, ms};
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    m->dm = keep;
    if (st != TMD_OK) return st;
    m->dm.tile_rows = top.tile_rows;
    m->dm.pair_bps = top.pair_blocks_per_sm;
    if (best) *best = top;
    return TMD_OK;
}

}  // namespace

extern "C" {

tmd_status tmd_autotune(tmd_model *m, tmd_nlist *nl, const double *pos, const int32_t *types, int64_t n,
                        const double box[3], tmd_tuning *best, tmd_stream_t stream) {
    g_err[0] = 0;
    if (!m || !nl || !nl->built || n < 1) { set_error("null model, unbuilt table or no atoms"); return TMD_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    tmd_status st;
    if ((st = grow(&nl->io_forces, &nl->cap_io_forces, 3 * n)) != TMD_OK) return st;
    if ((st = grow(&nl->io_red, &nl->cap_io_red, 16)) != TMD_OK) return st;
    return tune_shapes(m, s, best, [&]() {
        return run_compute(m, nl, pos, types, n, box, nl->io_red, nullptr, nl->io_forces, nl->io_red + 1, s);
    });
}

// --------------------------------------------------------------------- nlist
tmd_status tmd_nlist_create(tmd_nlist **out) {
    if (!out) { set_error("null output"); return TMD_ERR_INVALID_ARG; }
    *out = new (std::nothrow) tmd_nlist();
    if (!*out) { set_error("host allocation failed"); return TMD_ERR_OOM; }
    return TMD_OK;
}

tmd_status tmd_nlist_destroy(tmd_nlist *nl) {
    if (!nl) return TMD_OK;
    nlist_free(nl);
    delete nl;
    return TMD_OK;
}

tmd_status tmd_neighbors(const double *pos, const int32_t *types, int64_t n, const double box[3],
                         const int32_t pbc[3], double r_list, tmd_nlist *nl, tmd_stream_t stream) {
    g_err[0] = 0;
    if (!nl) { set_error("null neighbour table"); return TMD_ERR_INVALID_ARG; }
    tmd_status st = check_box(box, pbc);
    if (st != TMD_OK) return st;
    return build_neighbors(pos, types, n, box, pbc, r_list, nl, (cudaStream_t)stream);
}

tmd_status tmd_nlist_size(const tmd_nlist *nl, int64_t *n_atoms, int64_t *n_entries) {
    if (!nl || !nl->built) { set_error("neighbour table not built"); return TMD_ERR_INVALID_ARG; }
    if (n_atoms) *n_atoms = nl->n;
    if (n_entries) *n_entries = nl->nnz;
    return TMD_OK;
}

tmd_status tmd_nlist_export(const tmd_nlist *nl, int64_t *off, int32_t *nbr, int8_t *shift) {
    if (!nl || !nl->built) { set_error("neighbour table not built"); return TMD_ERR_INVALID_ARG; }
    TMD_CUDA(cudaDeviceSynchronize());
    const int64_t n = nl->n, nnz = nl->nnz;
    std::vector<int64_t> b((size_t)n), e((size_t)n);
    std::vector<int32_t> nb((size_t)std::max<int64_t>(nnz, 1));
    std::vector<char4> sh((size_t)std::max<int64_t>(nnz, 1));
    if (n > 0) {
        TMD_CUDA(cudaMemcpy(b.data(), nl->beg, sizeof(int64_t) * n, cudaMemcpyDeviceToHost));
        TMD_CUDA(cudaMemcpy(e.data(), nl->end, sizeof(int64_t) * n, cudaMemcpyDeviceToHost));
    }
    if (nnz > 0) {
        TMD_CUDA(cudaMemcpy(nb.data(), nl->nbr, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost));
        TMD_CUDA(cudaMemcpy(sh.data(), nl->shift, sizeof(char4) * nnz, cudaMemcpyDeviceToHost));
    }
    // CSR in atom order, each atom's entries sorted by (species of j, j, sx, sy, sz)
    std::vector<int64_t> o((size_t)n + 1, 0);
    for (int64_t i = 0; i < n; ++i) o[i + 1] = o[i] + (e[i] - b[i]);
    if (off) std::memcpy(off, o.data(), sizeof(int64_t) * (n + 1));
    std::vector<uint64_t> keys;
    for (int64_t i = 0; i < n; ++i) {
        keys.clear();
        for (int64_t c = b[i]; c < e[i]; ++c) {
            const char4 v = sh[c];
            keys.push_back(((uint64_t)(uint8_t)v.w << 60) | ((uint64_t)(uint32_t)nb[c] << 15) |
                           ((uint64_t)(v.x + 16) << 10) | ((uint64_t)(v.y + 16) << 5) | (uint64_t)(v.z + 16));
        }
        std::sort(keys.begin(), keys.end());
        for (size_t k = 0; k < keys.size(); ++k) {
            const uint64_t key = keys[k];
            const int64_t dst = o[i] + (int64_t)k;
            if (nbr) nbr[dst] = (int32_t)((key >> 15) & 0x1FFFFFFFFFFFull);
            if (shift) {
                shift[3 * dst] = (int8_t)((int)((key >> 10) & 31) - 16);
                shift[3 * dst + 1] = (int8_t)((int)((key >> 5) & 31) - 16);
                shift[3 * dst + 2] = (int8_t)((int)(key & 31) - 16);
            }
        }
    }
    return TMD_OK;
}

// --------------------------------------------------------------------- compute
tmd_status tmd_compute(const tmd_model *model, tmd_nlist *nl, const double *pos, const int32_t *types, int64_t n,
                       const double box[3], double *energy, float *e_atom, float *forces, double *virial,
                       tmd_stream_t stream) {
    g_err[0] = 0;
    if (!box) { set_error("null box"); return TMD_ERR_INVALID_ARG; }
    if (n > 0 && (!pos || !types)) { set_error("null pos/types"); return TMD_ERR_INVALID_ARG; }
    return run_compute(model, nl, pos, types, n, box, energy, e_atom, forces, virial, (cudaStream_t)stream);
}

tmd_status tmd_compute_owned(const tmd_model *model, tmd_nlist *nl, const double *pos, const int32_t *types, int64_t n,
                             int64_t n_owned, const double box[3], double *energy, float *e_atom, float *forces,
                             double *virial, tmd_stream_t stream) {
    g_err[0] = 0;
    if (!model || !nl || !box) { set_error("null model, table or box"); return TMD_ERR_INVALID_ARG; }
    return run_compute_owned(model, nl, pos, types, n, n_owned, box, energy, e_atom, forces, virial,
                             (cudaStream_t)stream);
}

tmd_status tmd_descriptors(const tmd_model *model, tmd_nlist *nl, const double *pos, const int32_t *types,
                           int64_t n, const double box[3], float *G, float *dEdG, tmd_stream_t stream) {
    g_err[0] = 0;
    if (!box || (n > 0 && (!pos || !types || !G))) { set_error("null box/pos/types/G"); return TMD_ERR_INVALID_ARG; }
    return run_descriptors(model, nl, pos, types, n, box, G, dEdG, (cudaStream_t)stream);
}

tmd_status tmd_compute_noalloc(const tmd_model *model, const int64_t *off, const int32_t *nbr, const int8_t *shift4,
                               int64_t nnz, const double *pos, const int32_t *types, int64_t n, const double box[3],
                               double *energy, float *e_atom, float *forces, double *virial, tmd_stream_t stream) {
    g_err[0] = 0;
    return run_compute_noalloc(model, off, nbr, shift4, nnz, pos, types, n, box, energy, e_atom, forces, virial,
                               (cudaStream_t)stream);
}

tmd_status tmd_evaluate_host(const tmd_model *model, tmd_nlist *nl, const double *pos_host, const int32_t *types_host,
                             int64_t n, const double box[3], const int32_t pbc[3], double *energy_host,
                             float *forces_host, double *virial_host, tmd_stream_t stream) {
    g_err[0] = 0;
    if (!model || !nl) { set_error("null model or neighbour table"); return TMD_ERR_INVALID_ARG; }
    tmd_status st = check_box(box, pbc);
    if (st != TMD_OK) return st;
    if (n < 0 || (n > 0 && (!pos_host || !types_host))) { set_error("bad n or null host arrays"); return TMD_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = grow(&nl->io_pos, &nl->cap_io_pos, 3 * n)) != TMD_OK) return st;
    if ((st = grow(&nl->io_types, &nl->cap_io_types, n)) != TMD_OK) return st;
    if ((st = grow(&nl->io_forces, &nl->cap_io_forces, 3 * n)) != TMD_OK) return st;
    if ((st = grow(&nl->io_red, &nl->cap_io_red, 10)) != TMD_OK) return st;
    if (n > 0) {
        TMD_CUDA(cudaMemcpyAsync(nl->io_pos, pos_host, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
        TMD_CUDA(cudaMemcpyAsync(nl->io_types, types_host, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    }
    if ((st = build_neighbors(nl->io_pos, nl->io_types, n, box, pbc, (double)model->dm.rc, nl, s)) != TMD_OK) return st;
    if ((st = run_compute(model, nl, nl->io_pos, nl->io_types, n, box, nl->io_red, nullptr, nl->io_forces,
                          nl->io_red + 1, s)) != TMD_OK)
        return st;
    if (energy_host) TMD_CUDA(cudaMemcpyAsync(energy_host, nl->io_red, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (virial_host) TMD_CUDA(cudaMemcpyAsync(virial_host, nl->io_red + 1, 9 * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (forces_host && n > 0)
        TMD_CUDA(cudaMemcpyAsync(forces_host, nl->io_forces, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, s));
    TMD_CUDA(cudaStreamSynchronize(s));
    return TMD_OK;
}

// --------------------------------------------------------------------- MD
tmd_status tmd_system_create(int64_t n, const double box[3], const int32_t pbc[3], double skin, tmd_system **out) {
    g_err[0] = 0;
    if (!out) { set_error("null output"); return TMD_ERR_INVALID_ARG; }
    *out = nullptr;
    tmd_status st = check_box(box, pbc);
    if (st != TMD_OK) return st;
    if (n < 1 || n >= (int64_t(1) << 28)) { set_error("n = %lld outside [1, 2^28)", (long long)n); return TMD_ERR_INVALID_ARG; }
    if (!(std::isfinite(skin) && skin >= 0.0)) { set_error("skin must be finite and >= 0"); return TMD_ERR_INVALID_ARG; }
    tmd_system *sys = new (std::nothrow) tmd_system();
    if (!sys) { set_error("host allocation failed"); return TMD_ERR_OOM; }
    sys->n = n;
    for (int x = 0; x < 3; ++x) { sys->box[x] = box[x]; sys->pbc[x] = pbc[x] ? 1 : 0; }
    sys->skin = skin;
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMalloc(&sys->pos, sizeof(double) * 3 * n);
    if (e == cudaSuccess) e = cudaMalloc(&sys->vel, sizeof(double) * 3 * n);
    if (e == cudaSuccess) e = cudaMalloc(&sys->pos_ref, sizeof(double) * 3 * n);
    if (e == cudaSuccess) e = cudaMalloc(&sys->inv_mass, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&sys->mass, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&sys->types, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&sys->forces, sizeof(float) * 3 * n);
    if (e == cudaSuccess) e = cudaMalloc(&sys->red, sizeof(double) * 32);
    if (e == cudaSuccess) e = cudaMallocHost(&sys->h_red, sizeof(double) * 32);
    if (e == cudaSuccess) e = cudaMemset(sys->vel, 0, sizeof(double) * 3 * n);
    if (e == cudaSuccess) e = cudaMemset(sys->forces, 0, sizeof(float) * 3 * n);
    if (e == cudaSuccess) e = cudaMemset(sys->red, 0, sizeof(double) * 32);
    if (e != cudaSuccess) {
        tmd_system_destroy(sys);
        cudaGetLastError();
        set_error("system allocation: %s", cudaGetErrorString(e));
        return TMD_ERR_OOM;
    }
    *out = sys;
    return TMD_OK;
}

tmd_status tmd_system_destroy(tmd_system *sys) {
    if (!sys) return TMD_OK;
    void *sp_[] = {sys->snap_pos, sys->snap_vel, sys->snap_forces, sys->run_flags};
    for (void *q : sp_)
        if (q) cudaFree(q);
    if (sys->h_run) cudaFreeHost(sys->h_run);
    void *p[] = {sys->pos, sys->vel, sys->pos_ref, sys->inv_mass, sys->mass, sys->types, sys->forces, sys->red,
                 sys->part};
    for (void *q : p)
        if (q) cudaFree(q);
    if (sys->h_red) cudaFreeHost(sys->h_red);
    nlist_free(&sys->nl);
    delete sys;
    return TMD_OK;
}

tmd_status tmd_system_set_state(tmd_system *sys, const double *pos, const double *vel, const int32_t *types,
                                const double *masses, int32_t on_device, tmd_stream_t stream) {
    g_err[0] = 0;
    if (!sys || !pos || !types) { set_error("null system, pos or types"); return TMD_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const int64_t n = sys->n;
    TMD_CUDA(cudaMemcpyAsync(sys->pos, pos, sizeof(double) * 3 * n, k, s));
    TMD_CUDA(cudaMemcpyAsync(sys->types, types, sizeof(int32_t) * n, k, s));
    if (vel) TMD_CUDA(cudaMemcpyAsync(sys->vel, vel, sizeof(double) * 3 * n, k, s));
    else TMD_CUDA(cudaMemsetAsync(sys->vel, 0, sizeof(double) * 3 * n, s));
    if (masses) {
        if (!on_device)
            for (int64_t i = 0; i < n; ++i)
                if (!(masses[i] > 0.0 && std::isfinite(masses[i]))) { set_error("mass[%lld] must be > 0", (long long)i); return TMD_ERR_INVALID_ARG; }
        TMD_CUDA(cudaMemcpyAsync(sys->mass, masses, sizeof(double) * n, k, s));
        TMD_LAUNCH("k_inv_mass", s, k_inv_mass<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sys->mass, sys->inv_mass, n));
        TMD_CUDA(cudaGetLastError());
    }
    if (!on_device) TMD_CUDA(cudaStreamSynchronize(s));  // host arrays may be pageable and reused
    sys->step = 0;
    sys->rebuilds = 0;
    sys->need_rebuild = 1;
    sys->have_forces = 0;
    return TMD_OK;
}

tmd_status tmd_system_get_state(const tmd_system *sys, double *pos, double *vel, float *forces, int32_t on_device,
                                tmd_stream_t stream) {
    if (!sys) { set_error("null system"); return TMD_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const int64_t n = sys->n;
    if (pos) TMD_CUDA(cudaMemcpyAsync(pos, sys->pos, sizeof(double) * 3 * n, k, s));
    if (vel) TMD_CUDA(cudaMemcpyAsync(vel, sys->vel, sizeof(double) * 3 * n, k, s));
    if (forces) TMD_CUDA(cudaMemcpyAsync(forces, sys->forces, sizeof(float) * 3 * n, k, s));
    TMD_CUDA(cudaStreamSynchronize(s));
    return TMD_OK;
}

// The system's split-position arrays when they have room for its atoms (the
// drift and the wrap then keep them current and the evaluation does not form
// them again), else null.
static float4 *split_hi(const tmd_system *sys) {
    return sys->nl.ph && sys->nl.pl && sys->nl.cap_ph >= sys->n && sys->nl.cap_pl >= sys->n ? sys->nl.ph : nullptr;
}
static float4 *split_lo(const tmd_system *sys) { return split_hi(sys) ? sys->nl.pl : nullptr; }

static tmd_status rebuild_only(const tmd_model *model, tmd_system *sys, cudaStream_t s) {
    tmd_status st;
    {
        const double r_list = (double)model->dm.rc + sys->skin;
        const int64_t n = sys->n;
        TMD_LAUNCH("k_wrap", s, k_wrap<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sys->pos, n, sys->box[0], sys->box[1],
                                                                                  sys->box[2], sys->pbc[0], sys->pbc[1],
                                                                                  sys->pbc[2], split_hi(sys),
                                                                                  split_lo(sys)));
        if ((st = build_neighbors(sys->pos, sys->types, sys->n, sys->box, sys->pbc, r_list, &sys->nl, s)) != TMD_OK)
            return st;
        TMD_CUDA(cudaMemcpyAsync(sys->pos_ref, sys->pos, sizeof(double) * 3 * sys->n, cudaMemcpyDeviceToDevice, s));
        sys->rebuilds++;
        sys->need_rebuild = 0;
    }
    return TMD_OK;
}

static tmd_status rebuild_and_compute(const tmd_model *model, tmd_system *sys, bool rebuild, cudaStream_t s) {
    tmd_status st;
    if (rebuild && (st = rebuild_only(model, sys, s)) != TMD_OK) return st;
    return run_compute(model, &sys->nl, sys->pos, sys->types, sys->n, sys->box, sys->red, nullptr, sys->forces,
                       sys->red + 1, s);
}

// One velocity-Verlet step with the table policy, deciding on the host
// (reads the skin flag back unless the cadence already asks for a rebuild).
static tmd_status step_eager(const tmd_model *model, tmd_system *sys, double dt_fs, int32_t rebuild_every,
                             cudaStream_t s) {
    tmd_status st;
    const int64_t n = sys->n;
    const unsigned nb = (unsigned)((n + 255) / 256);
    int32_t *flag = reinterpret_cast<int32_t *>(sys->red + 20);
    const double lim = 0.5 * sys->skin;
    TMD_CUDA(cudaMemsetAsync(flag, 0, sizeof(int32_t), s));
    float4 *const ph = split_hi(sys), *const pl = split_lo(sys);
    TMD_LAUNCH("k_vv_first", s, k_vv_first<<<nb, 256, 0, s>>>(sys->pos, sys->vel, sys->forces, sys->inv_mass, n,
                                                              dt_fs, sys->pos_ref, lim * lim, flag, ph, pl));
    TMD_CUDA(cudaGetLastError());
    sys->step++;
    bool rebuild = sys->need_rebuild || (rebuild_every > 0 && (sys->step % rebuild_every) == 0);
    if (!rebuild) {
        TMD_CUDA(cudaMemcpyAsync(sys->h_red + 20, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        TMD_CUDA(cudaStreamSynchronize(s));
        int32_t f = 0;
        std::memcpy(&f, sys->h_red + 20, sizeof(int32_t));
        rebuild = (f & 1) != 0;
    }
    if (rebuild && (st = rebuild_only(model, sys, s)) != TMD_OK) return st;
    if (rebuild) sys->near_skin = 0;
    // force evaluation and second half kick: one captured graph per table layout
    if ((st = reserve_compute(model->dm, &sys->nl, n, n)) != TMD_OK) return st;
    std::vector<uintptr_t> key;
    model_key(model, key);
    nlist_key(sys->nl, key);
    const void *sp[] = {sys->pos, sys->vel, sys->types, sys->forces, sys->red, sys->inv_mass};
    for (const void *q : sp) key.push_back((uintptr_t)q);
    key.push_back((uintptr_t)n);
    key.push_back(bits_of(dt_fs));
    key.push_back((uintptr_t)ph);
    for (int x = 0; x < 3; ++x) key.push_back(bits_of(sys->box[x]));
    return graphed(sys->g_step, key, s, [&]() {
        tmd_status st2 = run_compute(model, &sys->nl, sys->pos, sys->types, sys->n, sys->box, sys->red, nullptr,
                                     nullptr, sys->red + 1, s, ph != nullptr);
        if (st2 != TMD_OK) return st2;
        TMD_LAUNCH("k_vv_second", s, k_vv_second_fq<<<nb, 256, 0, s>>>(
                                         sys->vel, reinterpret_cast<const long long *>(sys->nl.Fq), sys->forces,
                                         sys->inv_mass, n, dt_fs));
        TMD_CUDA(cudaGetLastError());
        return TMD_OK;
    });
}

constexpr int RUN_MAX = 16;   // steps per launch sequence when no cadence sets the length

// k steps as one launch sequence with no host decision in between: the state
// is copied aside first; with a cadence the run starts on a cadence step,
// whose rebuild runs on the device (build_tables device_only), and every
// other step records its skin check in its own flag.  The flags, the table's
// entry counter and its status are read once at the end.  A run in which an
// atom moved more than skin / 2 before a rebuild was due, or whose table
// overflowed, is undone and stepped again on the host-decided path, so the
// trajectory is always the one that path gives.
static tmd_status step_run(const tmd_model *model, tmd_system *sys, double dt_fs, int k, bool rebuild_first,
                           cudaStream_t s, bool *redo) {
    tmd_status st;
    *redo = false;
    const int64_t n = sys->n;
    const unsigned nb = (unsigned)((n + 255) / 256);
    const double lim = 0.5 * sys->skin;
    if (!sys->snap_pos) {
        cudaError_t e = cudaMalloc(&sys->snap_pos, sizeof(double) * 3 * n);
        if (e == cudaSuccess) e = cudaMalloc(&sys->snap_vel, sizeof(double) * 3 * n);
        if (e == cudaSuccess) e = cudaMalloc(&sys->snap_forces, sizeof(float) * 3 * n);
        if (e == cudaSuccess) e = cudaMalloc(&sys->run_flags, sizeof(int32_t) * RUN_MAX);
        if (e == cudaSuccess) e = cudaMallocHost(&sys->h_run, sizeof(int64_t) * (RUN_MAX + 4));
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("run state: %s", cudaGetErrorString(e));
            return TMD_ERR_OOM;
        }
    }
    if ((st = reserve_compute(model->dm, &sys->nl, n, n)) != TMD_OK) return st;
    tmd_nlist *nl = &sys->nl;
    SysParams q;
    int64_t ncell = 0;
    if (rebuild_first &&
        (st = make_sys_params(sys->box, sys->pbc, (double)model->dm.rc + sys->skin, &q, &ncell)) != TMD_OK)
        return st;
    std::vector<uintptr_t> key;
    model_key(model, key);
    nlist_key(*nl, key);
    const void *sp[] = {sys->pos, sys->vel, sys->types, sys->forces, sys->red, sys->inv_mass, sys->snap_pos};
    for (const void *p : sp) key.push_back((uintptr_t)p);
    key.push_back((uintptr_t)n);
    key.push_back((uintptr_t)k);
    key.push_back((uintptr_t)rebuild_first);
    key.push_back(bits_of(dt_fs));
    key.push_back(bits_of(sys->skin));
    for (int x = 0; x < 3; ++x) key.push_back(bits_of(sys->box[x]));
    float4 *const ph = split_hi(sys), *const pl = split_lo(sys);
    key.push_back((uintptr_t)ph);
    st = graphed(sys->g_run, key, s, [&]() {
        TMD_CUDA(cudaMemcpyAsync(sys->snap_pos, sys->pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s));
        TMD_CUDA(cudaMemcpyAsync(sys->snap_vel, sys->vel, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s));
        TMD_CUDA(cudaMemcpyAsync(sys->snap_forces, sys->forces, sizeof(float) * 3 * n, cudaMemcpyDeviceToDevice, s));
        TMD_CUDA(cudaMemsetAsync(sys->run_flags, 0, sizeof(int32_t) * RUN_MAX, s));
        for (int j = 0; j < k; ++j) {
            TMD_LAUNCH("k_vv_first", s, k_vv_first<<<nb, 256, 0, s>>>(sys->pos, sys->vel, sys->forces, sys->inv_mass,
                                                                      n, dt_fs, sys->pos_ref, lim * lim,
                                                                      sys->run_flags + j, ph, pl));
            if (j == 0 && rebuild_first) {
                TMD_LAUNCH("k_wrap", s, k_wrap<<<nb, 256, 0, s>>>(sys->pos, n, sys->box[0], sys->box[1], sys->box[2],
                                                                  sys->pbc[0], sys->pbc[1], sys->pbc[2], ph, pl));
                tmd_status b = build_tables(sys->pos, sys->types, n, 1, &q, nullptr, nullptr, nullptr, ncell, nl, s,
                                            true);
                if (b != TMD_OK) return b;
                TMD_CUDA(cudaMemcpyAsync(sys->pos_ref, sys->pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s));
            }
            tmd_status c = run_compute(model, nl, sys->pos, sys->types, n, sys->box, sys->red, nullptr, nullptr,
                                       sys->red + 1, s, ph != nullptr);
            if (c != TMD_OK) return c;
            TMD_LAUNCH("k_vv_second", s, k_vv_second_fq<<<nb, 256, 0, s>>>(
                                             sys->vel, reinterpret_cast<const long long *>(nl->Fq), sys->forces,
                                             sys->inv_mass, n, dt_fs));
            TMD_CUDA(cudaGetLastError());
        }
        return TMD_OK;
    });
    if (st != TMD_OK) return st;
    TMD_CUDA(cudaMemcpyAsync(sys->h_run, sys->run_flags, sizeof(int32_t) * RUN_MAX, cudaMemcpyDeviceToHost, s));
    TMD_CUDA(cudaMemcpyAsync(sys->h_run + RUN_MAX / 2, nl->counter, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TMD_CUDA(cudaMemcpyAsync(sys->h_run + RUN_MAX / 2 + 1, nl->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    TMD_CUDA(cudaStreamSynchronize(s));
    int32_t flags[RUN_MAX];
    std::memcpy(flags, sys->h_run, sizeof(flags));
    bool moved = false, near = false;
    for (int j = rebuild_first ? 1 : 0; j < k; ++j) {
        moved = moved || (flags[j] & 1) != 0;
        near = near || (flags[j] & 2) != 0;
    }
    bool bad_table = false;
    if (rebuild_first) {
        int32_t status = 0;
        std::memcpy(&status, sys->h_run + RUN_MAX / 2 + 1, sizeof(int32_t));
        bad_table = sys->h_run[RUN_MAX / 2] > std::min(nl->cap_nnz, nl->cap_shift) || status != 0;
    }
    if (moved || bad_table) {   // undo: back to the state at the start of the run
        TMD_CUDA(cudaMemcpyAsync(sys->pos, sys->snap_pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s));
        TMD_CUDA(cudaMemcpyAsync(sys->vel, sys->snap_vel, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s));
        TMD_CUDA(cudaMemcpyAsync(sys->forces, sys->snap_forces, sizeof(float) * 3 * n, cudaMemcpyDeviceToDevice, s));
        if (bad_table) sys->need_rebuild = 1;   // the host-decided path rebuilds with room for every entry
        sys->reruns++;
        *redo = true;
        return TMD_OK;
    }
    if (rebuild_first) {
        sys->rebuilds++;
        sys->need_rebuild = 0;
    }
    // an atom came close to skin/2: step one at a time until the next rebuild
    // (instead of running ahead into a run that would be undone)
    sys->near_skin = near ? 1 : 0;
    sys->step += k;
    sys->runs++;
    return TMD_OK;
}

tmd_status tmd_step(const tmd_model *model, tmd_system *sys, double dt_fs, int32_t nsteps, int32_t rebuild_every,
                    tmd_thermo *thermo, tmd_stream_t stream) {
    g_err[0] = 0;
    if (!model || !sys) { set_error("null model or system"); return TMD_ERR_INVALID_ARG; }
    if (!(std::isfinite(dt_fs)) || nsteps < 0 || rebuild_every < 0) { set_error("bad dt/nsteps/rebuild_every"); return TMD_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    tmd_status st;
    const int64_t n = sys->n;
    if (!sys->have_forces) {
        if ((st = rebuild_and_compute(model, sys, true, s)) != TMD_OK) return st;
        sys->have_forces = 1;
    }
    // Runs of steps as one launch sequence where they are exact: with a
    // cadence, from a cadence step up to the step before the next one; with
    // the skin criterion alone, RUN_MAX steps at a time.  The rest, and every
    // run that had to be undone, step one at a time with the host reading the
    // skin flag.
    const bool runs = g_graphs && sys->skin > 0.0 && (rebuild_every == 0 || rebuild_every <= RUN_MAX);
    int it = 0;
    while (it < nsteps) {
        const int64_t next = sys->step + 1;
        int k = 0;
        bool rebuild_first = false;
        if (runs && !sys->need_rebuild && sys->nl.built && (!sys->near_skin || rebuild_every > 0)) {
            if (rebuild_every > 0 && next % rebuild_every == 0 && nsteps - it >= rebuild_every) {
                k = rebuild_every;
                rebuild_first = true;
            } else if (rebuild_every == 0 && nsteps - it >= 2) {
                k = std::min(RUN_MAX, nsteps - it);
            }
        }
        if (k > 0) {
            bool redo = false;
            if ((st = step_run(model, sys, dt_fs, k, rebuild_first, s, &redo)) != TMD_OK) return st;
            if (!redo) {
                it += k;
                continue;
            }
            for (int j = 0; j < k; ++j)
                if ((st = step_eager(model, sys, dt_fs, rebuild_every, s)) != TMD_OK) return st;
            it += k;
            continue;
        }
        if ((st = step_eager(model, sys, dt_fs, rebuild_every, s)) != TMD_OK) return st;
        ++it;
    }
    if (thermo) {
        const int kb = (int)std::min<int64_t>((n + 255) / 256, 1024);
        if ((st = grow(&sys->part, &sys->cap_part, 6 * (int64_t)kb)) != TMD_OK) return st;
        TMD_LAUNCH("k_kinetic", s, k_kinetic<<<kb, 256, 0, s>>>(sys->vel, sys->mass, n, sys->part));
        TMD_LAUNCH("k_kinetic_total", s, k_kinetic_total<<<1, 32, 0, s>>>(sys->part, kb, sys->red + 10));
        TMD_CUDA(cudaGetLastError());
        TMD_CUDA(cudaMemcpyAsync(sys->h_red, sys->red, sizeof(double) * 16, cudaMemcpyDeviceToHost, s));
        TMD_CUDA(cudaStreamSynchronize(s));
        const double *r = sys->h_red;
        const double conv = 1.0 / ACC_CONV;  // amu A^2/fs^2 -> eV
        const double mvv[9] = {r[10], r[13], r[14], r[13], r[11], r[15], r[14], r[15], r[12]};
        thermo->e_pot = r[0];
        thermo->e_kin = 0.5 * (r[10] + r[11] + r[12]) * conv;
        const double dof = n > 1 ? 3.0 * n - 3.0 : 3.0;
        thermo->temperature = 2.0 * thermo->e_kin / (dof * KB_EV);
        const double V = sys->box[0] * sys->box[1] * sys->box[2];
        for (int t = 0; t < 9; ++t) {
            thermo->virial[t] = r[1 + t];
            thermo->pressure[t] = (mvv[t] * conv + r[1 + t]) / V;
        }
        thermo->step = sys->step;
        thermo->rebuilds = sys->rebuilds;
    }
    return TMD_OK;
}

tmd_status tmd_system_counters(const tmd_system *sys, int64_t *steps, int64_t *rebuilds, int64_t *runs,
                               int64_t *reruns) {
    if (!sys) { set_error("null system"); return TMD_ERR_INVALID_ARG; }
    if (steps) *steps = sys->step;
    if (rebuilds) *rebuilds = sys->rebuilds;
    if (runs) *runs = sys->runs;
    if (reruns) *reruns = sys->reruns;
    return TMD_OK;
}

tmd_status tmd_step_host(const tmd_model *model, tmd_system *sys, double *pos_host, double *vel_host, float *forces_host,
                         double dt_fs, int32_t nsteps, int32_t rebuild_every, tmd_thermo *thermo, tmd_stream_t stream) {
    g_err[0] = 0;
    if (!model || !sys || !pos_host || !vel_host) { set_error("null model, system or host state"); return TMD_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = sys->n;
    TMD_CUDA(cudaMemcpyAsync(sys->pos, pos_host, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
    TMD_CUDA(cudaMemcpyAsync(sys->vel, vel_host, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
    if (forces_host) {
        TMD_CUDA(cudaMemcpyAsync(sys->forces, forces_host, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s));
        sys->have_forces = 1;
    } else {
        sys->have_forces = 0;
    }
    // no forced rebuild: the skin check compares the uploaded positions with
    // those of the last build, so positions the caller moved by more than
    // skin/2 (a wrap included) rebuild the table, and the cadence holds
    // across calls
    tmd_status st = tmd_step(model, sys, dt_fs, nsteps, rebuild_every, thermo, stream);
    if (st != TMD_OK) return st;
    TMD_CUDA(cudaMemcpyAsync(pos_host, sys->pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
    TMD_CUDA(cudaMemcpyAsync(vel_host, sys->vel, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
    if (forces_host) TMD_CUDA(cudaMemcpyAsync(forces_host, sys->forces, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, s));
    TMD_CUDA(cudaStreamSynchronize(s));
    return TMD_OK;
}


// --------------------------------------------------------------------- batches
}  // extern "C"

struct tmd_batch {
    int32_t S = 0;
    std::vector<int64_t> off;        // [S+1] atom offsets
    std::vector<double> box;         // [S][3]
    std::vector<int32_t> pbc;        // [S][3]
    std::vector<tmd::SysParams> sp;  // for the current list radius
    std::vector<int32_t> cell_off;
    int64_t ncell = 0;
    double r_list = -1.0;
    int64_t n = 0;
    double *pos = nullptr, *vel = nullptr, *mass = nullptr, *inv_mass = nullptr;
    int32_t *types = nullptr, *sys_of = nullptr;
    float *forces = nullptr, *e_atom = nullptr, *w_atom = nullptr;
    int64_t *d_off = nullptr;
    uint8_t *active = nullptr;       // [S] device flags
    int32_t *act_list = nullptr;     // [S] device list of active systems
    double *sys_out = nullptr;       // [S][16] device per-system sums
    double *h_out = nullptr;         // pinned mirror
    int32_t *h_act = nullptr;        // pinned staging of the active list
    uint8_t *h_flags = nullptr;      // pinned staging of the flags
    std::vector<uint8_t> has_forces;
    std::vector<int64_t> steps;
    // resident neighbour tables: every system's segments live in its own
    // region of one entry pool (pool.nbr / pool.shift, capacity pool_cap),
    // kept between calls and rebuilt per system
    double skin = 0.0;               // tables hold pairs within rc + skin
    int32_t rebuild_every = 0;       // cadence (0: the skin criterion only)
    tmd_nlist pool;                  // resident tables; perm = evaluation order of the active atoms
    tmd_nlist scratch;               // one build of the systems being rebuilt
    int64_t pool_cap = 0, pool_used = 0;
    std::vector<int64_t> rbase, rcap;                // region of each system (rcap 0: none)
    std::vector<std::pair<int64_t, int64_t>> holes;  // released regions (base, capacity)
    std::vector<uint8_t> built;      // table valid for the positions since its build
    std::vector<int64_t> rebuilds;
    std::vector<int64_t> species;    // [S][MAX_SPECIES] atoms per species
    double *pos_ref = nullptr;       // [n][3] positions at each system's last build
    int32_t *rank = nullptr;         // [n] index of an atom among its system's atoms of its species
    int32_t *d_moved = nullptr;      // [S] skin check
    int32_t *h_moved = nullptr;      // pinned mirror
    int64_t *d_region = nullptr;     // [S][2] region base, capacity
    unsigned long long *d_fill = nullptr;  // [S] entries placed per region
    int32_t *d_overflow = nullptr;
    unsigned long long *h_fill = nullptr;  // pinned: fill [S] then overflow
    int64_t *d_pbase = nullptr;      // [S][MAX_SPECIES] evaluation order blocks
    std::vector<int64_t> h_pbase;
    uint8_t *d_rflags = nullptr;     // [S] systems being rebuilt
    tmd::GraphCache g_eval, g_step;   // captured evaluation / evaluation + second half kick
};

namespace {

tmd_status batch_params(tmd_batch *b, double r_list) {
    if (b->r_list == r_list && !b->sp.empty()) return TMD_OK;
    std::vector<tmd::SysParams> sp(b->S);
    std::vector<int32_t> cell_off(b->S);
    int64_t total = 0;
    for (int k = 0; k < b->S; ++k) {
        int64_t nc = 0;
        tmd_status st = tmd::make_sys_params(&b->box[3 * k], &b->pbc[3 * k], r_list, &sp[k], &nc);
        if (st != TMD_OK) return st;
        sp[k].cell_off = (int)total;
        total += nc;
    }
    b->sp.swap(sp);
    b->cell_off.swap(cell_off);
    b->ncell = total;
    // a new list radius invalidates every resident table
    if (b->r_list != r_list)
        for (int k = 0; k < b->S; ++k) b->built[k] = 0;
    b->r_list = r_list;
    tmd_status st;
    if ((st = tmd::grow(&b->pool.sp, &b->pool.cap_sp, b->S)) != TMD_OK) return st;
    TMD_CUDA(cudaMemcpy(b->pool.sp, b->sp.data(), sizeof(tmd::SysParams) * b->S, cudaMemcpyHostToDevice));
    return TMD_OK;
}

// flags + list of the active systems to the device (pinned staging)
tmd_status batch_activate(tmd_batch *b, const int32_t *systems, int32_t n_act, cudaStream_t s, int64_t *atoms) {
    std::memset(b->h_flags, 0, b->S);
    int64_t na = 0;
    for (int k = 0; k < n_act; ++k) {
        const int32_t sys = systems[k];
        if (sys < 0 || sys >= b->S || b->h_flags[sys]) {
            tmd::set_error("active system %d out of range or repeated", sys);
            return TMD_ERR_INVALID_ARG;
        }
        b->h_flags[sys] = 1;
        b->h_act[k] = sys;
        na += b->off[sys + 1] - b->off[sys];
    }
    TMD_CUDA(cudaMemcpyAsync(b->active, b->h_flags, b->S, cudaMemcpyHostToDevice, s));
    TMD_CUDA(cudaMemcpyAsync(b->act_list, b->h_act, sizeof(int32_t) * n_act, cudaMemcpyHostToDevice, s));
    *atoms = na;
    return TMD_OK;
}

// ---- entry pool: one region per system, first fit over released regions
void region_free(tmd_batch *b, int k) {
    if (b->rcap[k] > 0) b->holes.push_back({b->rbase[k], b->rcap[k]});
    b->rbase[k] = 0;
    b->rcap[k] = 0;
    b->built[k] = 0;
}

tmd_status region_alloc(tmd_batch *b, int k, int64_t want, cudaStream_t s) {
    for (size_t h = 0; h < b->holes.size(); ++h)
        if (b->holes[h].second >= want) {
            b->rbase[k] = b->holes[h].first;
            b->rcap[k] = want;
            if (b->holes[h].second == want) b->holes.erase(b->holes.begin() + h);
            else b->holes[h] = {b->holes[h].first + want, b->holes[h].second - want};
            return TMD_OK;
        }
    if (b->pool_used + want > b->pool_cap) {
        // a larger pool keeps every region where it is (same entry offsets)
        const int64_t cap = std::max<int64_t>(b->pool_used + want, b->pool_cap + b->pool_cap / 2);
        int32_t *nbr = nullptr;
        char4 *sh = nullptr;
        cudaError_t e = cudaMalloc(&nbr, sizeof(int32_t) * cap);
        if (e == cudaSuccess) e = cudaMalloc(&sh, sizeof(char4) * cap);
        if (e != cudaSuccess) {
            if (nbr) cudaFree(nbr);
            cudaGetLastError();
            tmd::set_error("neighbour table pool of %lld entries: %s", (long long)cap, cudaGetErrorString(e));
            return TMD_ERR_OOM;
        }
        if (b->pool_used > 0) {
            TMD_CUDA(cudaMemcpyAsync(nbr, b->pool.nbr, sizeof(int32_t) * b->pool_used, cudaMemcpyDeviceToDevice, s));
            TMD_CUDA(cudaMemcpyAsync(sh, b->pool.shift, sizeof(char4) * b->pool_used, cudaMemcpyDeviceToDevice, s));
            TMD_CUDA(cudaStreamSynchronize(s));
        }
        if (b->pool.nbr) cudaFree(b->pool.nbr);
        if (b->pool.shift) cudaFree(b->pool.shift);
        b->pool.nbr = nbr;
        b->pool.shift = sh;
        b->pool.cap_nnz = b->pool.cap_shift = cap;
        b->pool_cap = cap;
        b->pool.nnz = cap;   // sizes the pair cache: one slot per pool entry
    }
    b->rbase[k] = b->pool_used;
    b->rcap[k] = want;
    b->pool_used += want;
    return TMD_OK;
}

// entries of system k from the uniform-density estimate, with headroom
int64_t region_estimate(const tmd_batch *b, int k, double r_list) {
    const double nk = (double)(b->off[k + 1] - b->off[k]);
    const double vol = b->box[3 * k] * b->box[3 * k + 1] * b->box[3 * k + 2];
    return (int64_t)(1.3 * nk * (nk / vol) * (4.0 / 3.0) * M_PI * r_list * r_list * r_list) + 64;
}

// Wrap and rebuild the tables of the systems flagged in rflags (host [S]):
// one build over their atoms (r_list = rc + skin) into the scratch table,
// whose segments then move to the systems' regions of the pool.
tmd_status batch_rebuild(const tmd_model *model, tmd_batch *b, const std::vector<uint8_t> &rflags, cudaStream_t s) {
    tmd_status st;
    const double r_list = (double)model->dm.rc + b->skin;
    if ((st = batch_params(b, r_list)) != TMD_OK) return st;
    std::vector<int64_t> nsys(b->S, 0);
    int64_t nr = 0;
    for (int k = 0; k < b->S; ++k)
        if (rflags[k]) {
            nsys[k] = b->off[k + 1] - b->off[k];
            nr += nsys[k];
        }
    if (nr == 0) return TMD_OK;
    std::memcpy(b->h_flags, rflags.data(), b->S);
    TMD_CUDA(cudaMemcpyAsync(b->d_rflags, b->h_flags, b->S, cudaMemcpyHostToDevice, s));
    const unsigned nb = (unsigned)((b->n + 255) / 256);
    TMD_LAUNCH("k_wrap_b", s, k_wrap_b<<<nb, 256, 0, s>>>(b->pos, b->n, b->pool.sp, b->sys_of, b->d_rflags));
    if ((st = tmd::build_tables(b->pos, b->types, b->n, b->S, b->sp.data(), b->sys_of, b->d_rflags, nsys.data(),
                                b->ncell, &b->scratch, s)) != TMD_OK)
        return st;
    // per-atom segment bounds of the pool cover every atom of the batch
    if ((st = tmd::grow(&b->pool.beg, &b->pool.cap_beg, b->n)) != TMD_OK) return st;
    if ((st = tmd::grow(&b->pool.end, &b->pool.cap_end, b->n)) != TMD_OK) return st;
    for (int k = 0; k < b->S; ++k)
        if (rflags[k] && b->rcap[k] == 0 && (st = region_alloc(b, k, region_estimate(b, k, r_list), s)) != TMD_OK)
            return st;
    for (int attempt = 0; attempt < 3; ++attempt) {
        std::vector<int64_t> reg(2 * (size_t)b->S);
        for (int k = 0; k < b->S; ++k) {
            reg[2 * k] = b->rbase[k];
            reg[2 * k + 1] = b->rcap[k];
        }
        TMD_CUDA(cudaMemcpyAsync(b->d_region, reg.data(), sizeof(int64_t) * 2 * b->S, cudaMemcpyHostToDevice, s));
        TMD_CUDA(cudaMemsetAsync(b->d_fill, 0, sizeof(unsigned long long) * b->S, s));
        TMD_CUDA(cudaMemsetAsync(b->d_overflow, 0, sizeof(int32_t), s));
        const unsigned cb = (unsigned)std::min<int64_t>((nr + 7) / 8, 65535);
        TMD_LAUNCH("k_region_copy", s, k_region_copy<<<cb, 256, 0, s>>>(
                                           b->scratch.beg, b->scratch.end, b->scratch.nbr, b->scratch.shift,
                                           b->scratch.perm, nr, b->sys_of, b->d_region, b->d_fill, b->pool.beg,
                                           b->pool.end, b->pool.nbr, b->pool.shift, b->d_overflow));
        TMD_CUDA(cudaGetLastError());
        TMD_CUDA(cudaMemcpyAsync(b->h_fill, b->d_fill, sizeof(unsigned long long) * b->S, cudaMemcpyDeviceToHost, s));
        TMD_CUDA(cudaMemcpyAsync(b->h_fill + b->S, b->d_overflow, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        TMD_CUDA(cudaStreamSynchronize(s));
        int32_t over = 0;
        std::memcpy(&over, b->h_fill + b->S, sizeof(int32_t));
        if (!over) break;
        if (attempt == 2) {
            tmd::set_error("neighbour table regions still too small after resizing");
            return TMD_ERR_CAPACITY;
        }
        // a region too small for its system: a new one with headroom
        for (int k = 0; k < b->S; ++k)
            if (rflags[k] && (int64_t)b->h_fill[k] > b->rcap[k]) {
                const int64_t want = (int64_t)b->h_fill[k] + (int64_t)b->h_fill[k] / 4 + 64;
                region_free(b, k);
                if ((st = region_alloc(b, k, want, s)) != TMD_OK) return st;
            }
    }
    TMD_LAUNCH("k_copy_ref_b", s, k_copy_ref_b<<<nb, 256, 0, s>>>(b->pos, b->pos_ref, b->n, b->sys_of, b->d_rflags));
    TMD_CUDA(cudaGetLastError());
    for (int k = 0; k < b->S; ++k)
        if (rflags[k]) {
            b->built[k] = 1;
            b->rebuilds[k]++;
        }
    b->pool.r_list = r_list;
    b->pool.built = 1;
    return TMD_OK;
}

// evaluation order of the active atoms (flags already on the device)
tmd_status batch_order(tmd_batch *b, int32_t n_act, cudaStream_t s) {
    tmd_status st;
    int64_t run = 0;
    for (int t = 0; t < TMD_MAX_SPECIES; ++t) {
        int64_t c = 0;
        for (int k = 0; k < n_act; ++k) {
            const int sys = b->h_act[k];
            b->h_pbase[(size_t)sys * TMD_MAX_SPECIES + t] = run + c;
            c += b->species[(size_t)sys * TMD_MAX_SPECIES + t];
        }
        b->pool.type_count[t] = (int32_t)c;
        run += c;
    }
    b->pool.n_active = run;
    if ((st = tmd::grow(&b->pool.perm, &b->pool.cap_perm, std::max<int64_t>(run, 1))) != TMD_OK) return st;
    TMD_CUDA(cudaMemcpyAsync(b->d_pbase, b->h_pbase.data(), sizeof(int64_t) * TMD_MAX_SPECIES * b->S,
                             cudaMemcpyHostToDevice, s));
    const unsigned nb = (unsigned)((b->n + 255) / 256);
    TMD_LAUNCH("k_eval_perm", s, k_eval_perm<<<nb, 256, 0, s>>>(b->n, b->sys_of, b->active, b->types, b->rank,
                                                                b->d_pbase, b->pool.perm));
    TMD_CUDA(cudaGetLastError());
    // the pageable h_pbase is read by the copy above before it is rewritten
    TMD_CUDA(cudaStreamSynchronize(s));
    return TMD_OK;
}

// tables for the active systems that have none (or all of them without a skin)
tmd_status batch_prepare(const tmd_model *model, tmd_batch *b, int32_t n_act, cudaStream_t s, bool all) {
    std::vector<uint8_t> rf(b->S, 0);
    for (int k = 0; k < n_act; ++k) {
        const int sys = b->h_act[k];
        if (all || b->skin <= 0.0 || !b->built[sys] || b->r_list != (double)model->dm.rc + b->skin) rf[sys] = 1;
    }
    return batch_rebuild(model, b, rf, s);
}

void batch_key(const tmd_model *model, const tmd_batch *b, int32_t n_act, std::vector<uintptr_t> &key) {
    model_key(model, key);
    nlist_key(b->pool, key);
    const void *bp[] = {b->pos, b->vel, b->mass, b->inv_mass, b->types, b->sys_of, b->forces, b->e_atom, b->w_atom,
                        b->d_off, b->active, b->act_list, b->sys_out};
    for (const void *q : bp) key.push_back((uintptr_t)q);
    key.push_back((uintptr_t)n_act);
    key.push_back((uintptr_t)b->n);
}

// evaluate the active systems on their current tables (captured graph when repeated)
tmd_status batch_compute_only(const tmd_model *model, tmd_batch *b, int32_t n_act, cudaStream_t s) {
    tmd_status st;
    if ((st = tmd::reserve_compute(model->dm, &b->pool, b->n, b->pool.n_active)) != TMD_OK) return st;
    std::vector<uintptr_t> key;
    batch_key(model, b, n_act, key);
    return graphed(b->g_eval, key, s, [&]() {
        return tmd::run_compute_batch(model, &b->pool, b->pos, b->types, b->n, b->sys_of, b->forces, b->e_atom,
                                      b->w_atom, b->act_list, n_act, b->d_off, b->vel, b->mass, b->sys_out, s);
    });
}

// tables where needed, evaluation order, evaluation (flags already set)
tmd_status batch_eval(const tmd_model *model, tmd_batch *b, int32_t n_act, cudaStream_t s) {
    tmd_status st;
    if ((st = batch_prepare(model, b, n_act, s, false)) != TMD_OK) return st;
    if ((st = batch_order(b, n_act, s)) != TMD_OK) return st;
    return batch_compute_only(model, b, n_act, s);
}

void batch_results(tmd_batch *b, int32_t n_act, double *energy, double *virial, tmd_thermo *thermo) {
    const double conv = 103.6427;  // amu A^2/fs^2 -> eV
    for (int k = 0; k < n_act; ++k) {
        const double *r = b->h_out + 16 * k;
        const int sys = b->h_act[k];
        if (energy) energy[k] = r[0];
        if (virial)
            for (int t = 0; t < 9; ++t) virial[9 * k + t] = r[1 + t];
        if (thermo) {
            tmd_thermo &th = thermo[k];
            const int64_t na = b->off[sys + 1] - b->off[sys];
            const double mvv[9] = {r[10], r[13], r[14], r[13], r[11], r[15], r[14], r[15], r[12]};
            th.e_pot = r[0];
            th.e_kin = 0.5 * (r[10] + r[11] + r[12]) * conv;
            const double dof = na > 1 ? 3.0 * na - 3.0 : 3.0;
            th.temperature = 2.0 * th.e_kin / (dof * KB_EV);
            const double V = b->box[3 * sys] * b->box[3 * sys + 1] * b->box[3 * sys + 2];
            for (int t = 0; t < 9; ++t) {
                th.virial[t] = r[1 + t];
                th.pressure[t] = (mvv[t] * conv + r[1 + t]) / V;
            }
            th.step = b->steps[sys];
            th.rebuilds = b->rebuilds[sys];
        }
    }
}

}  // namespace

extern "C" {

tmd_status tmd_batch_create(int32_t n_systems, const int64_t *n_atoms, const double *boxes, const int32_t *pbc,
                            tmd_batch **out) {
    g_err[0] = 0;
    if (!out || !n_atoms || !boxes || !pbc || n_systems < 1) { set_error("bad batch arguments"); return TMD_ERR_INVALID_ARG; }
    *out = nullptr;
    tmd_batch *b = new (std::nothrow) tmd_batch();
    if (!b) { set_error("host allocation failed"); return TMD_ERR_OOM; }
    b->S = n_systems;
    b->off.assign(n_systems + 1, 0);
    b->box.assign(boxes, boxes + 3 * (size_t)n_systems);
    b->pbc.assign(pbc, pbc + 3 * (size_t)n_systems);
    for (int k = 0; k < n_systems; ++k) {
        if (n_atoms[k] < 1) { delete b; set_error("system %d has no atoms", k); return TMD_ERR_INVALID_ARG; }
        tmd_status st = check_box(&boxes[3 * k], &pbc[3 * k]);
        if (st != TMD_OK) { delete b; return st; }
        b->off[k + 1] = b->off[k] + n_atoms[k];
    }
    b->n = b->off[n_systems];
    if (b->n >= (int64_t(1) << 28)) { delete b; set_error("too many atoms in the batch"); return TMD_ERR_INVALID_ARG; }
    b->has_forces.assign(n_systems, 0);
    b->steps.assign(n_systems, 0);
    b->built.assign(n_systems, 0);
    b->rebuilds.assign(n_systems, 0);
    b->rbase.assign(n_systems, 0);
    b->rcap.assign(n_systems, 0);
    b->species.assign((size_t)n_systems * TMD_MAX_SPECIES, 0);
    b->h_pbase.assign((size_t)n_systems * TMD_MAX_SPECIES, 0);
    const int64_t n = b->n;
    cudaError_t e = cudaMalloc(&b->pos, sizeof(double) * 3 * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->vel, sizeof(double) * 3 * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->mass, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->inv_mass, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->types, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->sys_of, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->forces, sizeof(float) * 3 * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->e_atom, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->w_atom, sizeof(float) * 9 * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_off, sizeof(int64_t) * (n_systems + 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->active, n_systems);
    if (e == cudaSuccess) e = cudaMalloc(&b->act_list, sizeof(int32_t) * n_systems);
    if (e == cudaSuccess) e = cudaMalloc(&b->sys_out, sizeof(double) * 16 * n_systems);
    if (e == cudaSuccess) e = cudaMalloc(&b->pos_ref, sizeof(double) * 3 * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->rank, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_moved, sizeof(int32_t) * n_systems);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_region, sizeof(int64_t) * 2 * n_systems);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_fill, sizeof(unsigned long long) * n_systems);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_overflow, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_pbase, sizeof(int64_t) * TMD_MAX_SPECIES * n_systems);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_rflags, n_systems);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_out, sizeof(double) * 16 * n_systems);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_act, sizeof(int32_t) * n_systems);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_flags, n_systems);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_moved, sizeof(int32_t) * n_systems);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_fill, sizeof(unsigned long long) * (n_systems + 1));
    if (e == cudaSuccess) e = cudaMemset(b->vel, 0, sizeof(double) * 3 * n);
    if (e == cudaSuccess) e = cudaMemset(b->forces, 0, sizeof(float) * 3 * n);
    if (e == cudaSuccess) e = cudaMemset(b->types, 0, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMemset(b->rank, 0, sizeof(int32_t) * n);
    if (e == cudaSuccess) {
        std::vector<int32_t> so((size_t)n);
        for (int k = 0; k < n_systems; ++k)
            for (int64_t i = b->off[k]; i < b->off[k + 1]; ++i) so[i] = k;
        e = cudaMemcpy(b->sys_of, so.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemcpy(b->d_off, b->off.data(), sizeof(int64_t) * (n_systems + 1), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        tmd_batch_destroy(b);
        cudaGetLastError();
        set_error("batch allocation: %s", cudaGetErrorString(e));
        return TMD_ERR_OOM;
    }
    for (int k = 0; k < n_systems; ++k)   // until set_system: every atom species 0
        b->species[(size_t)k * TMD_MAX_SPECIES] = b->off[k + 1] - b->off[k];
    *out = b;
    return TMD_OK;
}

tmd_status tmd_batch_destroy(tmd_batch *b) {
    if (!b) return TMD_OK;
    void *p[] = {b->pos, b->vel, b->mass, b->inv_mass, b->types, b->sys_of, b->forces, b->e_atom, b->w_atom,
                 b->d_off, b->active, b->act_list, b->sys_out, b->pos_ref, b->rank, b->d_moved, b->d_region,
                 b->d_fill, b->d_overflow, b->d_pbase, b->d_rflags};
    for (void *q : p)
        if (q) cudaFree(q);
    void *hp[] = {b->h_out, b->h_act, b->h_flags, b->h_moved, b->h_fill};
    for (void *q : hp)
        if (q) cudaFreeHost(q);
    nlist_free(&b->pool);
    nlist_free(&b->scratch);
    delete b;
    return TMD_OK;
}

tmd_status tmd_batch_set_system(tmd_batch *b, int32_t sys, const double *pos, const double *vel, const int32_t *types,
                                const double *masses, tmd_stream_t stream) {
    g_err[0] = 0;
    if (!b || sys < 0 || sys >= b->S || !pos || !types || !masses) { set_error("bad arguments"); return TMD_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t o = b->off[sys], n = b->off[sys + 1] - o;
    for (int64_t i = 0; i < n; ++i)
        if (!(masses[i] > 0.0 && std::isfinite(masses[i]))) { set_error("mass[%lld] must be > 0", (long long)i); return TMD_ERR_INVALID_ARG; }
    // per-species counts and each atom's rank among its species (evaluation order)
    std::vector<int32_t> rank((size_t)n);
    int64_t cnt[TMD_MAX_SPECIES] = {};
    for (int64_t i = 0; i < n; ++i) {
        if (types[i] < 0 || types[i] >= TMD_MAX_SPECIES) {
            set_error("types[%lld] = %d outside [0, %d)", (long long)i, types[i], TMD_MAX_SPECIES);
            return TMD_ERR_INVALID_ARG;
        }
        rank[i] = (int32_t)cnt[types[i]]++;
    }
    TMD_CUDA(cudaMemcpyAsync(b->pos + 3 * o, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
    TMD_CUDA(cudaMemcpyAsync(b->types + o, types, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    TMD_CUDA(cudaMemcpyAsync(b->mass + o, masses, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    TMD_CUDA(cudaMemcpyAsync(b->rank + o, rank.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    if (vel) TMD_CUDA(cudaMemcpyAsync(b->vel + 3 * o, vel, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
    else TMD_CUDA(cudaMemsetAsync(b->vel + 3 * o, 0, sizeof(double) * 3 * n, s));
    TMD_LAUNCH("k_inv_mass", s, k_inv_mass<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(b->mass + o, b->inv_mass + o, n));
    TMD_CUDA(cudaGetLastError());
    TMD_CUDA(cudaStreamSynchronize(s));  // host arrays may be pageable and reused
    for (int t = 0; t < TMD_MAX_SPECIES; ++t) b->species[(size_t)sys * TMD_MAX_SPECIES + t] = cnt[t];
    b->has_forces[sys] = 0;
    b->steps[sys] = 0;
    b->rebuilds[sys] = 0;
    b->built[sys] = 0;   // new positions: the table is built again (in its region) before use
    return TMD_OK;
}

tmd_status tmd_batch_get_system(const tmd_batch *b, int32_t sys, double *pos, double *vel, float *forces,
                                tmd_stream_t stream) {
    if (!b || sys < 0 || sys >= b->S) { set_error("bad arguments"); return TMD_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t o = b->off[sys], n = b->off[sys + 1] - o;
    if (pos) TMD_CUDA(cudaMemcpyAsync(pos, b->pos + 3 * o, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
    if (vel) TMD_CUDA(cudaMemcpyAsync(vel, b->vel + 3 * o, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
    if (forces) TMD_CUDA(cudaMemcpyAsync(forces, b->forces + 3 * o, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, s));
    TMD_CUDA(cudaStreamSynchronize(s));
    return TMD_OK;
}

tmd_status tmd_batch_set_skin(tmd_batch *b, double skin, int32_t rebuild_every) {
    g_err[0] = 0;
    if (!b || !(std::isfinite(skin) && skin >= 0.0) || rebuild_every < 0) {
        set_error("bad arguments: skin must be finite and >= 0, rebuild_every >= 0");
        return TMD_ERR_INVALID_ARG;
    }
    if (skin != b->skin)
        for (int k = 0; k < b->S; ++k) b->built[k] = 0;
    b->skin = skin;
    b->rebuild_every = rebuild_every;
    return TMD_OK;
}

tmd_status tmd_batch_release(tmd_batch *b, int32_t sys) {
    g_err[0] = 0;
    if (!b || sys < 0 || sys >= b->S) { set_error("bad arguments"); return TMD_ERR_INVALID_ARG; }
    region_free(b, sys);
    return TMD_OK;
}

tmd_status tmd_batch_table_info(const tmd_batch *b, int32_t sys, int64_t *region_entries, int64_t *pool_entries,
                                int64_t *rebuilds) {
    if (!b || sys < 0 || sys >= b->S) { set_error("bad arguments"); return TMD_ERR_INVALID_ARG; }
    if (region_entries) *region_entries = b->rcap[sys];
    if (pool_entries) *pool_entries = b->pool_cap;
    if (rebuilds) *rebuilds = b->rebuilds[sys];
    return TMD_OK;
}

tmd_status tmd_batch_compute(const tmd_model *model, tmd_batch *b, const int32_t *systems, int32_t n_act,
                             double *energy, double *virial, tmd_stream_t stream) {
    g_err[0] = 0;
    if (!model || !b || !systems || n_act < 1 || n_act > b->S) { set_error("bad arguments"); return TMD_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    int64_t na = 0;
    tmd_status st;
    if ((st = batch_activate(b, systems, n_act, s, &na)) != TMD_OK) return st;
    if ((st = batch_eval(model, b, n_act, s)) != TMD_OK) return st;
    TMD_CUDA(cudaMemcpyAsync(b->h_out, b->sys_out, sizeof(double) * 16 * n_act, cudaMemcpyDeviceToHost, s));
    TMD_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < n_act; ++k) b->has_forces[systems[k]] = 1;
    batch_results(b, n_act, energy, virial, nullptr);
    return TMD_OK;
}

tmd_status tmd_batch_step(const tmd_model *model, tmd_batch *b, const int32_t *systems, int32_t n_act, double dt_fs,
                          int32_t nsteps, tmd_thermo *thermo, tmd_stream_t stream) {
    g_err[0] = 0;
    if (!model || !b || !systems || n_act < 1 || n_act > b->S || nsteps < 0 || !std::isfinite(dt_fs)) {
        set_error("bad arguments");
        return TMD_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int64_t na = 0;
    tmd_status st;
    if ((st = batch_activate(b, systems, n_act, s, &na)) != TMD_OK) return st;
    bool need_init = false;
    for (int k = 0; k < n_act; ++k) need_init = need_init || !b->has_forces[systems[k]] || !b->built[systems[k]];
    if (need_init) {  // initial forces (systems that have them and a table are recomputed identically)
        std::vector<uint8_t> rf(b->S, 0);
        for (int k = 0; k < n_act; ++k)
            if (!b->has_forces[systems[k]] || !b->built[systems[k]]) rf[systems[k]] = 1;
        if ((st = batch_rebuild(model, b, rf, s)) != TMD_OK) return st;
        if ((st = batch_order(b, n_act, s)) != TMD_OK) return st;
        if ((st = batch_compute_only(model, b, n_act, s)) != TMD_OK) return st;
        for (int k = 0; k < n_act; ++k) b->has_forces[systems[k]] = 1;
    } else if ((st = batch_order(b, n_act, s)) != TMD_OK) {
        return st;
    }
    const unsigned nb = (unsigned)((b->n + 255) / 256);
    const bool skin = b->skin > 0.0;
    const double lim = 0.5 * b->skin;
    std::vector<uint8_t> rf(b->S);
    for (int it = 0; it < nsteps; ++it) {
        if (skin) TMD_CUDA(cudaMemsetAsync(b->d_moved, 0, sizeof(int32_t) * b->S, s));
        TMD_LAUNCH("k_vv_first_b", s, k_vv_first_b<<<nb, 256, 0, s>>>(b->pos, b->vel, b->forces, b->inv_mass, b->n,
                                                                      dt_fs, b->sys_of, b->active, b->pos_ref,
                                                                      lim * lim, skin ? b->d_moved : nullptr));
        TMD_CUDA(cudaGetLastError());
        for (int k = 0; k < n_act; ++k) b->steps[systems[k]]++;
        // which tables to rebuild: without a skin every step; else on the
        // cadence, or when an atom of the system moved more than skin / 2
        // (the skin criterion, read back once per step)
        std::fill(rf.begin(), rf.end(), 0);
        if (skin) {
            TMD_CUDA(cudaMemcpyAsync(b->h_moved, b->d_moved, sizeof(int32_t) * b->S, cudaMemcpyDeviceToHost, s));
            TMD_CUDA(cudaStreamSynchronize(s));
        }
        for (int k = 0; k < n_act; ++k) {
            const int sys = systems[k];
            const bool due = b->rebuild_every > 0 && (b->steps[sys] % b->rebuild_every) == 0;
            if (!skin || due || b->h_moved[sys] || !b->built[sys]) rf[sys] = 1;
        }
        if ((st = batch_rebuild(model, b, rf, s)) != TMD_OK) return st;
        // evaluation and second half kick: one captured graph per table layout
        if ((st = tmd::reserve_compute(model->dm, &b->pool, b->n, b->pool.n_active)) != TMD_OK) return st;
        std::vector<uintptr_t> key;
        batch_key(model, b, n_act, key);
        key.push_back(bits_of(dt_fs));
        st = graphed(b->g_step, key, s, [&]() {
            tmd_status st2 = tmd::run_compute_batch(model, &b->pool, b->pos, b->types, b->n, b->sys_of, b->forces,
                                                    b->e_atom, b->w_atom, b->act_list, n_act, b->d_off, b->vel,
                                                    b->mass, b->sys_out, s);
            if (st2 != TMD_OK) return st2;
            TMD_LAUNCH("k_vv_second_b", s, k_vv_second_b<<<nb, 256, 0, s>>>(b->vel, b->forces, b->inv_mass, b->n,
                                                                            dt_fs, b->sys_of, b->active));
            TMD_CUDA(cudaGetLastError());
            return TMD_OK;
        });
        if (st != TMD_OK) return st;
    }
    if (thermo || nsteps == 0) {
        // kinetic terms after the second half kick
        TMD_LAUNCH("k_sys_reduce", s, tmd::sys_reduce_launch(b->act_list, n_act, b->d_off, b->e_atom, b->w_atom, b->vel,
                                                             b->mass, b->sys_out, s));
    }
    TMD_CUDA(cudaMemcpyAsync(b->h_out, b->sys_out, sizeof(double) * 16 * n_act, cudaMemcpyDeviceToHost, s));
    TMD_CUDA(cudaStreamSynchronize(s));
    batch_results(b, n_act, nullptr, nullptr, thermo);
    return TMD_OK;
}

tmd_status tmd_batch_autotune(tmd_model *m, tmd_batch *b, const int32_t *systems, int32_t n_act, tmd_tuning *best,
                              tmd_stream_t stream) {
    g_err[0] = 0;
    if (!m || !b || !systems || n_act < 1 || n_act > b->S) { set_error("bad arguments"); return TMD_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    int64_t na = 0;
    tmd_status st;
    if ((st = batch_activate(b, systems, n_act, s, &na)) != TMD_OK) return st;
    if ((st = batch_eval(m, b, n_act, s)) != TMD_OK) return st;   // tables of the listed systems
    return tune_shapes(m, s, best, [&]() {
        return tmd::run_compute_batch(m, &b->pool, b->pos, b->types, b->n, b->sys_of, b->forces, b->e_atom, b->w_atom,
                                      b->act_list, n_act, b->d_off, b->vel, b->mass, b->sys_out, s);
    });
}

}  // extern "C"
