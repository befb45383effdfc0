// In-cutoff screening of the neighbour table (Sec. "The Tensor Formalism",
// the setup of D_abcx and R_abc before the H and M tensors; the cutoff rule
// "r >= r_cutoff is forced to zero"): for every atom, the entries of its table
// segment (built with rc + skin) that lie within rc, compacted in table order
// into the pair cache read by the descriptor and force passes.
//
// The descriptor pass used to screen the entries itself, one warp per atom,
// with every chunk's position gathers on its critical path.  Screening is
// cheap arithmetic over gathered data, so it runs here on its own with few
// registers and many warps in flight, which hides the latency of the table
// reads and position gathers; the passes behind it stream the compacted
// pairs.
#include <algorithm>

#include "pair_kernels.cuh"

namespace tmd {

namespace {

constexpr int SCREEN_WARPS = 8;

// One warp per atom (perm order), 32 table entries per step.  Few registers
// keep many warps resident, which is what hides the latency of the dependent
// reads (segment bounds, table entries, neighbour positions).
__global__ void __launch_bounds__(SCREEN_WARPS * 32, 6) k_screen(DevNlist nl, float rc2h, float rc2l) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t nw = (int64_t)gridDim.x * SCREEN_WARPS;
    for (int64_t p = (int64_t)blockIdx.x * SCREEN_WARPS + (threadIdx.x >> 5); p < nl.n; p += nw) {
        const int a = nl.perm[p];
        const int64_t beg = nl.beg[a], end = nl.end[a];
        const float4 ih = nl.ph[a], il = nl.pl[a];
        float Lh[3], Ll[3];
        pair_box(nl, a, Lh, Ll);
        int kept = 0;
        for (int64_t base = beg; base < end; base += 32) {
            const int64_t c = base + lane;
            bool v = false;
            float4 e;
            float2 e2;
            if (c < end) {
                const int j = nl.nbr[c];
                const char4 s = nl.shift[c];
                const float4 jh = nl.ph[j], jl = nl.pl[j];
                float dx, dy, dz, r2h, r2l;
                pair_geom(jh, jl, ih, il, s, Lh, Ll, dx, dy, dz, r2h, r2l);
                v = (r2h < rc2h) || (r2h == rc2h && r2l < rc2l);
                e = make_float4(dx, dy, dz, __uint_as_float((uint32_t)j | ((uint32_t)s.w << 28)));
                e2 = make_float2(r2h, r2l);
            }
            const unsigned m = __ballot_sync(0xffffffffu, v);
            if (v) {   // compacted in table order at [beg, beg + kept)
                const int64_t o = beg + kept + __popc(m & lt);
                nl.pq[o] = e;
                nl.pq2[o] = e2;
            }
            kept += __popc(m);
        }
        if (lane == 0) nl.npair[a] = kept;
    }
}

}  // namespace

tmd_status launch_screen(const DevModel &dm, const DevNlist &dn, cudaStream_t s) {
    if (dn.n == 0) return TMD_OK;
    if (!dn.pq || !dn.pq2 || !dn.npair) {
        set_error("screening needs the pair cache");
        return TMD_ERR_INVALID_ARG;
    }
    static int resident = 0;   // blocks of k_screen the GPU holds at once
    if (!resident) {
        int dev = 0, nsm = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        TMD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_screen, SCREEN_WARPS * 32, 0));
        resident = std::max(1, nsm) * std::max(1, per_sm);
    }
    const int64_t want = (dn.n + SCREEN_WARPS - 1) / SCREEN_WARPS;
    const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)resident));
    TMD_LAUNCH("k_screen", s, k_screen<<<nb, SCREEN_WARPS * 32, 0, s>>>(dn, dm.rc2h, dm.rc2l));
    TMD_CUDA(cudaGetLastError());
    return TMD_OK;
}

}  // namespace tmd
