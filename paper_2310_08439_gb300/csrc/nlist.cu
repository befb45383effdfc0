// Device cell list and neighbour table (the neighbour tensor R_abc of the
// paper's Sec. "The Tensor Formalism", built by binning with a skin buffer as
// in Sec. "Evaluation").
//
// Layout: atoms are binned into cells of side >= r_list; each atom's
// candidates come from the (2R+1)^3 stencil of unwrapped cells around its own,
// so periodic images (including self-images in boxes shorter than 2 r_list)
// are enumerated as distinct (cell, shift) pairs.  Candidates are screened in
// FP32 from a cell-sorted float4 copy of the positions; only pairs inside a
// rounding band around r_list^2 are decided in FP64 with the exact
// expression ((x_j + s L) - x_i), (dx^2 + dy^2) + dz^2, no FMA, which makes the
// table bit-identical to the plain definition.  The table is built in one
// pass: k_nbr_cell stages a cell's whole stencil in shared memory and screens
// it for all the cell's atoms at once (lane = atom, candidates broadcast, one
// hit bit per candidate), reserves room for the cell's atoms with one
// atomicAdd on a global counter and writes each atom's contiguous segment
// [beg[i], end[i]); atoms of cells whose stencil does not fit take the
// per-atom pass k_nbr.  Atom ids are sorted inside every cell first, so the
// entry order of each atom (stencil order, ascending id within a cell) is
// deterministic.
#include <cmath>
#include <cstring>

#include "tmd_internal.cuh"

namespace tmd {

namespace {

constexpr int BIN_THREADS = 256;
constexpr int NBR_WARPS = 4;
// per-block species counts: rows of TB_STRIDE ints (the species, then
// padding), two aligned int4 per row
constexpr int TB_STRIDE = 8;
static_assert(TMD_MAX_SPECIES <= TB_STRIDE, "species counts fit a row");

// cell index of each atom of an active system (global cell = the system's
// first cell + local cell), cell occupancy counts (stored at start[c+1]), per
// block species counts; flags atoms outside their box and bad species.  Atoms
// of inactive systems get cell -1 and are skipped by the later passes.
__global__ void k_bin(const double *__restrict__ pos, const int32_t *__restrict__ types, int64_t n,
                      const SysParams *__restrict__ sp, const int32_t *__restrict__ sys_of,
                      const uint8_t *__restrict__ active, int32_t *__restrict__ cell_of,
                      int32_t *__restrict__ cell_start, int32_t *__restrict__ type_block,
                      int32_t *__restrict__ status) {
    __shared__ int32_t s_cnt[TMD_MAX_SPECIES];
    if (threadIdx.x < TMD_MAX_SPECIES) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int t = -1;
    if (i < n) {
        const int sys = sys_of ? sys_of[i] : 0;
        if (active && !active[sys]) {
            cell_of[i] = -1;
        } else {
            const SysParams &q = sp[sys];
            const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
            const int bad = !(x >= 0.0 && x < q.L[0] && y >= 0.0 && y < q.L[1] && z >= 0.0 && z < q.L[2]);
            int cx = (int)(x * q.ic[0]), cy = (int)(y * q.ic[1]), cz = (int)(z * q.ic[2]);
            cx = min(max(cx, 0), q.nc[0] - 1);
            cy = min(max(cy, 0), q.nc[1] - 1);
            cz = min(max(cz, 0), q.nc[2] - 1);
            if (bad) atomicOr(status, DEV_ERR_OUTSIDE_BOX);
            const int c = q.cell_off + cx + q.nc[0] * (cy + q.nc[1] * cz);
            cell_of[i] = c;
            atomicAdd(&cell_start[c + 1], 1);
            t = types[i];
            if (t < 0 || t >= TMD_MAX_SPECIES) {
                atomicOr(status, DEV_ERR_BAD_TYPE);
                t = -1;
            }
        }
    }
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 0; s < TMD_MAX_SPECIES; ++s) {
        const unsigned m = __ballot_sync(0xffffffffu, t == s);
        if (lane == 0 && m) atomicAdd(&s_cnt[s], __popc(m));
    }
    __syncthreads();
    if (threadIdx.x < TMD_MAX_SPECIES) type_block[blockIdx.x * TB_STRIDE + threadIdx.x] = s_cnt[threadIdx.x];
}

// exclusive scan of the per-block species counts; writes the species start
// offsets type_start[0..MAX_SPECIES].
__global__ void __launch_bounds__(128) k_type_scan(int32_t *__restrict__ type_block, int nblocks,
                                                  int32_t *__restrict__ type_start) {
    // exclusive scan over the binning blocks, every species at once: thread t
    // owns a contiguous run of blocks (sums it, block-wide scan of the run
    // totals, then writes its run's offsets)
    constexpr int NS = TMD_MAX_SPECIES;
    __shared__ int32_t s_tot[128][NS];
    const int t = threadIdx.x;
    const int per = (nblocks + 127) / 128;
    const int b0 = min(nblocks, t * per), b1 = min(nblocks, b0 + per);
    int4 *rows = reinterpret_cast<int4 *>(type_block);   // two int4 per block
    int sum[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) sum[s] = 0;
    for (int b = b0; b < b1; ++b) {
        const int4 lo = rows[2 * (size_t)b], hi = rows[2 * (size_t)b + 1];
        const int v[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
        for (int s = 0; s < NS; ++s) sum[s] += v[s];
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) s_tot[t][s] = sum[s];
    __syncthreads();
    if (t < 32) {   // scan of the 128 run totals: 4 per lane, then across lanes
        int r[4][NS], acc[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) acc[s] = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                r[q][s] = acc[s];
                acc[s] += s_tot[4 * t + q][s];
            }
        int x[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) x[s] = acc[s];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1)
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const int y = __shfl_up_sync(0xffffffffu, x[s], d);
                if (t >= d) x[s] += y;
            }
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int s = 0; s < NS; ++s) s_tot[4 * t + q][s] = (x[s] - acc[s]) + r[q][s];
        if (t == 31) {   // x = the species totals
            int run = 0;
            type_start[0] = 0;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                run += x[s];
                type_start[s + 1] = run;
            }
        }
    }
    __syncthreads();
    int run[TB_STRIDE];
#pragma unroll
    for (int s = 0; s < TB_STRIDE; ++s) run[s] = s < NS ? s_tot[t][s] : 0;
    for (int b = b0; b < b1; ++b) {
        const int4 lo = rows[2 * (size_t)b], hi = rows[2 * (size_t)b + 1];
        const int v[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
        rows[2 * (size_t)b] = make_int4(run[0], run[1], run[2], run[3]);
        rows[2 * (size_t)b + 1] = make_int4(run[4], run[5], run[6], run[7]);
#pragma unroll
        for (int s = 0; s < NS; ++s) run[s] += v[s];
    }
}

// scatter atom ids into cells (order within a cell fixed by k_cell_sort) and
// stably into species order (perm).
__global__ void k_fill(const double *__restrict__ pos, const int32_t *__restrict__ types, int64_t n,
                       const int32_t *__restrict__ cell_of, const int32_t *__restrict__ cell_start,
                       int32_t *__restrict__ cell_fill, int32_t *__restrict__ cell_atoms,
                       const int32_t *__restrict__ type_block,
                       const int32_t *__restrict__ type_start, int32_t *__restrict__ perm) {
    __shared__ int32_t s_warp[BIN_THREADS / 32][TMD_MAX_SPECIES];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int t = -1;
    if (i < n && cell_of[i] >= 0) {
        t = types[i];
        if (t < 0 || t >= TMD_MAX_SPECIES) t = -1;
        const int c = cell_of[i];
        const int slot = cell_start[c] + atomicAdd(&cell_fill[c], 1);
        cell_atoms[slot] = (int32_t)i;
    }
    // stable species partition: rank = (earlier warps of the block) + (earlier lanes)
    unsigned masks[TMD_MAX_SPECIES];
#pragma unroll
    for (int s = 0; s < TMD_MAX_SPECIES; ++s) {
        masks[s] = __ballot_sync(0xffffffffu, t == s);
        if (lane == 0) s_warp[warp][s] = __popc(masks[s]);
    }
    __syncthreads();
    if (t >= 0) {
        int before = 0;
        for (int w = 0; w < warp; ++w) before += s_warp[w][t];
        before += __popc(masks[t] & ((1u << lane) - 1u));
        perm[type_start[t] + type_block[blockIdx.x * TB_STRIDE + t] + before] = (int32_t)i;
    }
}

constexpr int CELL_SORT_WARPS = 4;
constexpr int MAX_CELL = 1024;

// Sort the ids of every cell ascending (one warp per cell) and write the
// cell-sorted FP32 positions with the species in the top 4 bits of the id.
__global__ void __launch_bounds__(CELL_SORT_WARPS * 32)
    k_cell_sort(const int32_t *__restrict__ cell_start, int64_t ncell, int32_t *__restrict__ cell_atoms,
                const double *__restrict__ pos, const int32_t *__restrict__ types, float4 *__restrict__ cell_pos,
                int32_t *__restrict__ status) {
    __shared__ int32_t s_ids[CELL_SORT_WARPS][MAX_CELL];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t total = (int64_t)gridDim.x * CELL_SORT_WARPS;
    for (int64_t c = (int64_t)blockIdx.x * CELL_SORT_WARPS + warp; c < ncell; c += total) {
        const int beg = cell_start[c], cnt = cell_start[c + 1] - beg;
        if (cnt <= 32) {
            int v = lane < cnt ? cell_atoms[beg + lane] : 0x7fffffff;
#pragma unroll
            for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
                for (int j = k >> 1; j > 0; j >>= 1) {
                    const int w = __shfl_xor_sync(0xffffffffu, v, j);
                    const bool up = (lane & k) == 0, lower = (lane & j) == 0;
                    v = (lower == up) ? min(v, w) : max(v, w);
                }
            if (lane < cnt) cell_atoms[beg + lane] = v;
        } else if (cnt <= MAX_CELL) {
            int32_t *ids = s_ids[warp];
            for (int t = lane; t < cnt; t += 32) ids[t] = cell_atoms[beg + t];
            __syncwarp();
            for (int t = lane; t < cnt; t += 32) {  // rank sort (ids are distinct)
                const int e = ids[t];
                int rank = 0;
                for (int u = 0; u < cnt; ++u) rank += ids[u] < e;
                cell_atoms[beg + rank] = e;
            }
            __syncwarp();
        } else {
            if (lane == 0) atomicOr(status, DEV_ERR_CELL);
        }
        __syncwarp();
        for (int t = lane; t < cnt; t += 32) {
            const int i = cell_atoms[beg + t];
            int tt = types[i];
            tt = (tt < 0 || tt >= TMD_MAX_SPECIES) ? 0 : tt;
            cell_pos[beg + t] = make_float4((float)pos[3 * (int64_t)i], (float)pos[3 * (int64_t)i + 1],
                                            (float)pos[3 * (int64_t)i + 2],
                                            __int_as_float((int)((uint32_t)i | ((uint32_t)tt << 28))));
        }
    }
}

// cell index of u on one axis with its image shift (no division: |u| is
// within a few boxes of the range)
__device__ __forceinline__ int wrap_cell(int u, int nc, int &k) {
    int s = 0;
    k = u;
    while (k < 0) { k += nc; --s; }
    while (k >= nc) { k -= nc; ++s; }
    return s;
}

struct NbrParams {
    const int32_t *todo;  // per-atom pass: atoms to list (nullptr = all n)
    const unsigned long long *todo_n;  // per-atom pass: their count on the device (nullptr = n)
    const double *pos;
    const int32_t *cell_of;
    const int32_t *cell_start;
    const float4 *cell_pos;
    const SysParams *sp;
    const int32_t *sys_of;
    int64_t n;
    int64_t *beg, *end;   // per-atom segment of the table
    int32_t *nbr;
    char4 *shift;
    unsigned long long *counter;  // entries reserved so far
    int64_t cap;          // capacity of nbr / shift
    int32_t *status;
};

__device__ __forceinline__ uint64_t make_key(int t, int j, int sx, int sy, int sz) {
    return ((uint64_t)t << 60) | ((uint64_t)(uint32_t)j << 15) | ((uint64_t)(sx + 16) << 10) |
           ((uint64_t)(sy + 16) << 5) | (uint64_t)(sz + 16);
}

// The exact FP64 decision for a candidate inside the FP32 rounding band: the
// definition's expression, evaluated without FMA.  Kept out of line so that the
// compiler cannot predicate this (rarely needed) FP64 work onto every candidate.
__device__ __noinline__ bool exact_inside(const double *__restrict__ pos, int j, int sx, int sy, int sz, double xi,
                                          double yi, double zi, double L0, double L1, double L2, double r2) {
    const double ex = __dsub_rn(__dadd_rn(pos[3 * (int64_t)j], __dmul_rn((double)sx, L0)), xi);
    const double ey = __dsub_rn(__dadd_rn(pos[3 * (int64_t)j + 1], __dmul_rn((double)sy, L1)), yi);
    const double ez = __dsub_rn(__dadd_rn(pos[3 * (int64_t)j + 2], __dmul_rn((double)sz, L2)), zi);
    const double e2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
    return e2 < r2;
}

// Reserve room for one atom's entries (one atomicAdd) and write its segment.
__device__ __forceinline__ void emit_entries(const NbrParams &p, int64_t i, const uint64_t *keys, int count, int lane) {
    if (count > TMD_MAX_DEGREE) {
        if (lane == 0) {
            atomicOr(p.status, DEV_ERR_DEGREE);
            p.beg[i] = 0;
            p.end[i] = 0;
        }
        return;
    }
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(p.counter, (unsigned long long)count);
    base = __shfl_sync(0xffffffffu, base, 0);
    __syncwarp();
    if ((int64_t)base + count <= p.cap) {
        for (int c = lane; c < count; c += 32) {
            const uint64_t key = keys[c];
            const int t = (int)(key >> 60);
            const int j = (int)((key >> 15) & 0x1FFFFFFFFFFFull);
            const int sx = (int)((key >> 10) & 31) - 16, sy = (int)((key >> 5) & 31) - 16, sz = (int)(key & 31) - 16;
            p.nbr[base + c] = j;
            p.shift[base + c] = make_char4((signed char)sx, (signed char)sy, (signed char)sz, (signed char)t);
        }
    }
    if (lane == 0) {
        p.beg[i] = (int64_t)base;
        p.end[i] = (int64_t)base + count;
    }
}

// Per-atom pass (one warp per atom walks its own stencil): used for the atoms
// of cells whose stencil is too large for the cell-cooperative pass.
__device__ __forceinline__ void nbr_atom(const NbrParams &p, int64_t w, uint64_t *keys, int lane) {
    const int64_t i = p.todo ? (int64_t)p.todo[w] : w;
    const int cg = p.cell_of[i];
    if (cg < 0) {  // atom of an inactive system
        if (lane == 0) { p.beg[i] = 0; p.end[i] = 0; }
        return;
    }
    const SysParams &sysp = p.sp[p.sys_of ? p.sys_of[i] : 0];
    const int nc0 = sysp.nc[0], nc1 = sysp.nc[1], nc2 = sysp.nc[2];
    const double xi = p.pos[3 * i], yi = p.pos[3 * i + 1], zi = p.pos[3 * i + 2];
    const float xh = (float)xi, yh = (float)yi, zh = (float)zi;
    const int ci = cg - sysp.cell_off;
    const int cx = ci % nc0, cy = (ci / nc0) % nc1, cz = ci / (nc0 * nc1);
    const unsigned lt = (1u << lane) - 1u;
    int count = 0;
    for (int dz = -sysp.R[2]; dz <= sysp.R[2]; ++dz) {
        const int uz = cz + dz;
        if (!sysp.pbc[2] && (uz < 0 || uz >= nc2)) continue;
        int kz;
        const int sz = wrap_cell(uz, nc2, kz);
        const float zs = zh - (float)sz * sysp.Lh[2];
        for (int dy = -sysp.R[1]; dy <= sysp.R[1]; ++dy) {
            const int uy = cy + dy;
            if (!sysp.pbc[1] && (uy < 0 || uy >= nc1)) continue;
            int ky;
            const int sy = wrap_cell(uy, nc1, ky);
            const float ys = yh - (float)sy * sysp.Lh[1];
            const int row = sysp.cell_off + nc0 * (ky + nc1 * kz);
            int dx = -sysp.R[0];
            while (dx <= sysp.R[0]) {
                const int ux = cx + dx;
                if (!sysp.pbc[0] && (ux < 0 || ux >= nc0)) { ++dx; continue; }
                int kx;
                const int sx = wrap_cell(ux, nc0, kx);
                int len = 1;  // run of consecutive cells with the same shift
                while (dx + len <= sysp.R[0] && kx + len < nc0) ++len;
                const float xs = xh - (float)sx * sysp.Lh[0];
                const int beg = p.cell_start[row + kx], end = p.cell_start[row + kx + len];
                const bool self_img = (sx == 0 && sy == 0 && sz == 0);
                for (int b = beg; b < end; b += 32) {
                    const int q = b + lane;
                    bool in = false, band = false;
                    int j = 0, tj = 0;
                    if (q < end) {
                        const float4 cp = p.cell_pos[q];
                        const uint32_t w = (uint32_t)__float_as_int(cp.w);
                        j = (int)(w & 0x0FFFFFFFu);
                        tj = (int)(w >> 28);
                        const float ddx = cp.x - xs, ddy = cp.y - ys, ddz = cp.z - zs;
                        const float d2 = ddx * ddx + ddy * ddy + ddz * ddz;
                        in = d2 < sysp.r2lo;
                        band = !in && d2 < sysp.r2hi;
                    }
                    // rounding band: exact FP64 decision, reached through a
                    // warp-uniform branch and an out-of-line call so that the
                    // (rare) FP64 work is not predicated onto every candidate.
                    if (__any_sync(0xffffffffu, band)) {
                        if (band) in = exact_inside(p.pos, j, sx, sy, sz, xi, yi, zi, sysp.L[0], sysp.L[1], sysp.L[2], sysp.r2);
                    }
                    if (self_img && j == (int)i) in = false;
                    const unsigned m = __ballot_sync(0xffffffffu, in);
                    if (in) {
                        const int slot = count + __popc(m & lt);
                        if (slot < TMD_MAX_DEGREE) keys[slot] = make_key(tj, j, sx, sy, sz);
                    }
                    count += __popc(m);
                }
                dx += len;
            }
        }
    }
    emit_entries(p, i, keys, count, lane);
}

// One warp per atom, over a grid-stride loop: the count comes from the host
// (p.n) or, when the host has not read it, from the device (p.todo_n).
__global__ void __launch_bounds__(NBR_WARPS * 32) k_nbr(NbrParams p) {
    extern __shared__ uint64_t s_keys[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n = p.todo_n ? (int64_t)*p.todo_n : p.n;
    for (int64_t w = (int64_t)blockIdx.x * NBR_WARPS + warp; w < n; w += (int64_t)gridDim.x * NBR_WARPS)
        nbr_atom(p, w, s_keys + (size_t)warp * TMD_MAX_DEGREE, lane);
}

// Cell-cooperative pass: one block per cell stages the cell's whole stencil
// (cell-sorted candidates, image-shifted, FP32) in shared memory once; its
// warps then test each of the cell's atoms against the staged set.  The
// candidate order (stencil rows, runs, ascending ids) is the per-atom pass's,
// so both produce identical entries.  Cells whose stencil exceeds the staging
// capacity hand their atoms to the per-atom pass through `todo`.
constexpr int CELL_WARPS = 8;
constexpr int CAND_CAP = 1920;   // staged candidates per cell (60 groups of 32)
constexpr int LIST_CAP = 256;    // per-warp list of one atom's hits (longer lists: slower path)
constexpr int MAX_SEGS = 125;  // stencil cells ((2R+1)^3 for R <= 2; wider stencils take the per-atom pass)


// small integer -> float without a conversion instruction (|v| < 2^22):
// 1.5 * 2^23 + v has v in the low significand bits.
__device__ __forceinline__ float small_int_to_float(int v) {
    return __int_as_float(0x4B400000 + v) - 12582912.0f;
}

// The stencil of cell c as one segment per stencil cell, in (dz, dy, dx)
// order: first atom in cell order, count and shift code (all threads of the
// block; nothing when the stencil exceeds MAX_SEGS).
__device__ __forceinline__ void cell_lookup(const NbrParams &p, int64_t c, const int32_t *__restrict__ cell_sys,
                                            int *seg_b0, int *seg_cnt, uint16_t *seg_code) {
    const SysParams &sysp = p.sp[cell_sys ? cell_sys[c] : 0];
    const int nc0 = sysp.nc[0], nc1 = sysp.nc[1], nc2 = sysp.nc[2];
    const int w0 = 2 * sysp.R[0] + 1, w1 = 2 * sysp.R[1] + 1;
    const int nseg = w0 * w1 * (2 * sysp.R[2] + 1);
    if (nseg > MAX_SEGS) return;
    const int ci = (int)(c - sysp.cell_off);
    const int cx = ci % nc0, cy = (ci / nc0) % nc1, cz = ci / (nc0 * nc1);
    for (int t = threadIdx.x; t < nseg; t += blockDim.x) {
        const int tx = t % w0, tyz = t / w0;
        const int ux = cx + tx - sysp.R[0], uy = cy + tyz % w1 - sysp.R[1], uz = cz + tyz / w1 - sysp.R[2];
        int b0 = 0, cnt = 0, code = 0;
        if ((sysp.pbc[0] || (ux >= 0 && ux < nc0)) && (sysp.pbc[1] || (uy >= 0 && uy < nc1)) &&
            (sysp.pbc[2] || (uz >= 0 && uz < nc2))) {
            int kx, ky, kz;
            const int sx = wrap_cell(ux, nc0, kx);
            const int sy = wrap_cell(uy, nc1, ky);
            const int sz = wrap_cell(uz, nc2, kz);
            const int cell = sysp.cell_off + kx + nc0 * (ky + nc1 * kz);
            b0 = p.cell_start[cell];
            cnt = p.cell_start[cell + 1] - b0;
            code = (sx + 16) | ((sy + 16) << 5) | ((sz + 16) << 10);
        }
        seg_b0[t] = b0;
        seg_cnt[t] = cnt;
        seg_code[t] = (uint16_t)code;
    }
}

__device__ __forceinline__ void cp_async16_nbr(void *smem, const void *gmem) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem));
}

__global__ void __launch_bounds__(CELL_WARPS * 32)
    k_nbr_cell(NbrParams p, int64_t ncell, const int32_t *__restrict__ cell_sys,
               const int32_t *__restrict__ cell_atoms, int32_t *__restrict__ todo,
               unsigned long long *__restrict__ todo_count) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *cand = reinterpret_cast<float4 *>(smem_raw);                               // [CAND_CAP]
    char4 *cand_sh = reinterpret_cast<char4 *>(cand + CAND_CAP);                       // [CAND_CAP]
    // hit words of the current 32 atoms, [atom][group] (row padded by one word)
    uint32_t(*bits)[CAND_CAP / 32 + 1] = reinterpret_cast<uint32_t(*)[CAND_CAP / 32 + 1]>(cand_sh + CAND_CAP);
    // stencil segments, double-buffered: the next cell's are looked up while
    // this cell is processed; positions among the candidates for this cell
    __shared__ int s_seg_b0[2][MAX_SEGS], s_seg_cnt[2][MAX_SEGS], s_seg_pos[MAX_SEGS];
    __shared__ uint16_t s_seg_code[2][MAX_SEGS];
    __shared__ int s_total;
    __shared__ uint16_t s_list[CELL_WARPS][LIST_CAP];
    __shared__ int s_cnt[32];
    __shared__ int64_t s_off[32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned lt = (1u << lane) - 1u;
    int par = 0;
    if (blockIdx.x < ncell) cell_lookup(p, blockIdx.x, cell_sys, s_seg_b0[0], s_seg_cnt[0], s_seg_code[0]);
    for (int64_t c = blockIdx.x; c < ncell; c += gridDim.x, par ^= 1) {
        __syncthreads();   // this cell's segments are in place; the previous cell is done
        if (c + gridDim.x < ncell)
            cell_lookup(p, c + gridDim.x, cell_sys, s_seg_b0[par ^ 1], s_seg_cnt[par ^ 1], s_seg_code[par ^ 1]);
        const int abeg = p.cell_start[c], na = p.cell_start[c + 1] - abeg;
        if (na == 0) continue;  // uniform across the block
        const SysParams &sysp = p.sp[cell_sys ? cell_sys[c] : 0];
        const int w0 = 2 * sysp.R[0] + 1, w1 = 2 * sysp.R[1] + 1;
        const int nseg = w0 * w1 * (2 * sysp.R[2] + 1);
        if (nseg > MAX_SEGS) {  // wide stencil: per-atom pass
            for (int q = tid; q < na; q += blockDim.x) todo[atomicAdd(todo_count, 1ull)] = cell_atoms[abeg + q];
            continue;
        }
        const int *seg_b0 = s_seg_b0[par], *seg_cnt = s_seg_cnt[par];
        const uint16_t *seg_code = s_seg_code[par];
        if (warp == 0) {  // exclusive scan of the segments' candidate counts
            int run = 0;
            for (int r0 = 0; r0 < nseg; r0 += 32) {
                const int r = r0 + lane;
                const int v = r < nseg ? seg_cnt[r] : 0;
                int x = v;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, x, d);
                    if (lane >= d) x += y;
                }
                if (r < nseg) s_seg_pos[r] = run + x - v;
                run += __shfl_sync(0xffffffffu, x, 31);
            }
            if (lane == 0) s_total = run;
        }
        __syncthreads();
        const int total = s_total;
        if (total > CAND_CAP) {
            for (int q = tid; q < na; q += blockDim.x) todo[atomicAdd(todo_count, 1ull)] = cell_atoms[abeg + q];
            continue;
        }
        // stage the stencil in candidate order: every copy issued at once
        // (cp.async), then each stencil cell's image shift applied in place:
        // positions (x + sx Lx, y + sy Ly, z + sz Lz, id | species << 28) and
        // the table entry's shift (sx, sy, sz, species)
        for (int t = warp; t < nseg; t += CELL_WARPS) {
            const int cnt = seg_cnt[t], b0 = seg_b0[t], pos0 = s_seg_pos[t];
            for (int q = lane; q < cnt; q += 32) cp_async16_nbr(&cand[pos0 + q], &p.cell_pos[b0 + q]);
        }
        asm volatile("cp.async.commit_group;\n" ::);
        asm volatile("cp.async.wait_all;\n" ::);
        __syncthreads();
        for (int t = warp; t < nseg; t += CELL_WARPS) {
            const int cnt = seg_cnt[t];
            if (cnt == 0) continue;
            const int pos0 = s_seg_pos[t], code = seg_code[t];
            const int sx = (code & 31) - 16, sy = ((code >> 5) & 31) - 16, sz = ((code >> 10) & 31) - 16;
            const float ox = small_int_to_float(sx) * sysp.Lh[0];
            const float oy = small_int_to_float(sy) * sysp.Lh[1];
            const float oz = small_int_to_float(sz) * sysp.Lh[2];
            for (int q = lane; q < cnt; q += 32) {
                const float4 cp = cand[pos0 + q];
                cand[pos0 + q] = make_float4(cp.x + ox, cp.y + oy, cp.z + oz, cp.w);
                cand_sh[pos0 + q] = make_char4((signed char)sx, (signed char)sy, (signed char)sz,
                                               (signed char)((uint32_t)__float_as_int(cp.w) >> 28));
            }
        }
        __syncthreads();
        // the cell's own atoms: the centre segment (zero shift)
        const int qself = s_seg_pos[(sysp.R[2] * w1 + sysp.R[1]) * w0 + sysp.R[0]];
        const int ngroup = (total + 31) >> 5;

        for (int a0 = 0; a0 < na; a0 += 32) {
            // screen: lane = atom of the cell, candidates broadcast from shared
            // memory; bit k of a group word marks candidate 32 g + k inside r_list
            const int ai = a0 + lane;
            const bool act = ai < na;
            const float4 ip = act ? p.cell_pos[abeg + ai] : make_float4(3.0e18f, 3.0e18f, 3.0e18f, 0.f);
            for (int gi = warp; gi < ngroup; gi += CELL_WARPS) {   // candidate groups interleaved over warps
                const int qb = gi * 32;
                // the sign of d2 - r2 is the comparison; each candidate shifts
                // one bit in from the right, so candidate k ends at bit 31 - k
                uint32_t in_rev = 0, band_rev = 0;
#pragma unroll 8
                for (int k = 0; k < 32; ++k) {
                    const float4 cp = cand[qb + k];
                    const float ddx = cp.x - ip.x, ddy = cp.y - ip.y, ddz = cp.z - ip.z;
                    const float d2 = ddx * ddx + ddy * ddy + ddz * ddz;
                    in_rev = __funnelshift_l((uint32_t)__float_as_int(d2 - sysp.r2lo), in_rev, 1);
                    band_rev = __funnelshift_l((uint32_t)__float_as_int(d2 - sysp.r2hi), band_rev, 1);
                }
                uint32_t in_bits = __brev(in_rev), band_bits = __brev(band_rev);
                const uint32_t valid = (total - qb >= 32) ? 0xffffffffu : ((1u << (total - qb)) - 1u);
                in_bits &= valid;
                band_bits &= valid & ~in_bits;
                if (__any_sync(0xffffffffu, band_bits != 0)) {
                    // inside the FP32 rounding band: the exact FP64 decision
                    if (band_bits) {
                        const int i = cell_atoms[abeg + ai];
                        const double xi = p.pos[3 * (int64_t)i], yi = p.pos[3 * (int64_t)i + 1], zi = p.pos[3 * (int64_t)i + 2];
                        uint32_t bb = band_bits;
                        while (bb) {
                            const int k = __ffs(bb) - 1;
                            bb &= bb - 1;
                            const int q = qb + k;
                            const int j = (int)((uint32_t)__float_as_int(cand[q].w) & 0x0FFFFFFFu);
                            const char4 sh = cand_sh[q];
                            if (exact_inside(p.pos, j, sh.x, sh.y, sh.z, xi, yi, zi, sysp.L[0], sysp.L[1], sysp.L[2], sysp.r2))
                                in_bits |= 1u << k;
                        }
                    }
                }
                if (act && ((qself + ai) >> 5) == gi) in_bits &= ~(1u << ((qself + ai) & 31));  // (i, i, 0)
                if (act) bits[ai - a0][gi] = in_bits;
            }
            __syncthreads();
            // write-out.  Counts first (warp per atom, lane per candidate group),
            // then one reservation for the whole cell, then the entries.
            const int nact = min(32, na - a0);
            for (int aj = warp; aj < nact; aj += CELL_WARPS) {
                const uint32_t wd0 = lane < ngroup ? bits[aj][lane] : 0u;
                const uint32_t wd1 = lane + 32 < ngroup ? bits[aj][lane + 32] : 0u;
                const int count = __reduce_add_sync(0xffffffffu, __popc(wd0) + __popc(wd1));
                if (lane == 0) s_cnt[aj] = count;
            }
            __syncthreads();
            if (warp == 0) {   // exclusive scan of the counts and one atomicAdd for the cell
                int c = lane < nact ? s_cnt[lane] : 0;
                if (c > TMD_MAX_DEGREE) {
                    atomicOr(p.status, DEV_ERR_DEGREE);
                    c = 0;
                    s_cnt[lane] = -1;
                }
                int x = c;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, x, d);
                    if (lane >= d) x += y;
                }
                unsigned long long cb = 0;
                if (lane == 31) cb = atomicAdd(p.counter, (unsigned long long)x);
                cb = __shfl_sync(0xffffffffu, cb, 31);
                if (lane < nact) s_off[lane] = (int64_t)cb + (x - c);
            }
            __syncthreads();
            for (int aj = warp; aj < nact; aj += CELL_WARPS) {
                const int i = cell_atoms[abeg + a0 + aj];
                const int count = s_cnt[aj];
                if (count < 0) {   // over the degree limit: empty segment, status set
                    if (lane == 0) {
                        p.beg[i] = 0;
                        p.end[i] = 0;
                    }
                    continue;
                }
                const int64_t base = s_off[aj];
                const uint32_t wd0 = lane < ngroup ? bits[aj][lane] : 0u;
                const uint32_t wd1 = lane + 32 < ngroup ? bits[aj][lane + 32] : 0u;
                if (base + count <= p.cap && count <= LIST_CAP) {
                    // expand the words into the warp's list of candidate indices
                    // (lane per group, groups in order), then write the entries
                    // with consecutive lanes on consecutive entries
                    const int c0 = __popc(wd0);
                    int x0 = c0, x1 = __popc(wd1);
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const int y0 = __shfl_up_sync(0xffffffffu, x0, d), y1 = __shfl_up_sync(0xffffffffu, x1, d);
                        if (lane >= d) { x0 += y0; x1 += y1; }
                    }
                    uint16_t *list = s_list[warp];
                    int e = x0 - c0;
                    for (uint32_t wd = wd0; wd; wd &= wd - 1) list[e++] = (uint16_t)(lane * 32 + __ffs(wd) - 1);
                    e = __shfl_sync(0xffffffffu, x0, 31) + x1 - __popc(wd1);
                    for (uint32_t wd = wd1; wd; wd &= wd - 1) list[e++] = (uint16_t)((lane + 32) * 32 + __ffs(wd) - 1);
                    __syncwarp();
                    for (int k = lane; k < count; k += 32) {
                        const int q = list[k];
                        p.nbr[base + k] = (int)((uint32_t)__float_as_int(cand[q].w) & 0x0FFFFFFFu);
                        p.shift[base + k] = cand_sh[q];
                    }
                    __syncwarp();
                } else if (base + count <= p.cap) {
                    // long lists: groups in order, lane k takes bit k
                    int off = 0;
                    for (int gi = 0; gi < ngroup; ++gi) {
                        const uint32_t wd = bits[aj][gi];
                        if (wd == 0u) continue;
                        if ((wd >> lane) & 1u) {
                            const int q = gi * 32 + lane;
                            const int64_t ei = base + off + __popc(wd & lt);
                            p.nbr[ei] = (int)((uint32_t)__float_as_int(cand[q].w) & 0x0FFFFFFFu);
                            p.shift[ei] = cand_sh[q];
                        }
                        off += __popc(wd);
                    }
                }
                if (lane == 0) {
                    p.beg[i] = base;
                    p.end[i] = base + count;
                }
            }
            __syncthreads();
        }
    }
}

// system of every cell (batched builds)
__global__ void k_cell_sys(const SysParams *__restrict__ sp, int n_sys, int32_t *__restrict__ cell_sys) {
    const int k = blockIdx.y;
    if (k >= n_sys) return;
    const int c0 = sp[k].cell_off, nc = sp[k].nc[0] * sp[k].nc[1] * sp[k].nc[2];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) cell_sys[c0 + c] = k;
}

// ---------------------------------------------------------------- scans
template <typename T>
__global__ void k_scan_block(T *__restrict__ data, int64_t n, T *__restrict__ block_sums) {
    // inclusive scan of 2048-element chunks, 1024 threads x 2 items
    __shared__ T s_w[32];
    const int64_t base = (int64_t)blockIdx.x * 2048;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t i0 = base + 2 * tid;
    T a = (i0 < n) ? data[i0] : T(0);
    T b = (i0 + 1 < n) ? data[i0 + 1] : T(0);
    b += a;
    T v = b;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T u = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += u;
    }
    if (lane == 31) s_w[warp] = v;
    __syncthreads();
    if (warp == 0) {
        T w = s_w[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const T u = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += u;
        }
        s_w[lane] = w;
    }
    __syncthreads();
    const T pre = (warp > 0 ? s_w[warp - 1] : T(0)) + v - b;  // exclusive prefix of this thread
    if (i0 < n) data[i0] = pre + a;
    if (i0 + 1 < n) data[i0 + 1] = pre + b;
    if (tid == 1023 && block_sums) block_sums[blockIdx.x] = s_w[31];
}

template <typename T>
__global__ void k_scan_add(T *__restrict__ data, int64_t n, const T *__restrict__ block_sums) {
    const int64_t blk = blockIdx.x + 1;  // block 0 needs no offset
    const T add = block_sums[blk - 1];
    const int64_t base = blk * 2048;
    for (int t = threadIdx.x; t < 2048; t += blockDim.x) {
        const int64_t idx = base + t;
        if (idx < n) data[idx] += add;
    }
}

template <typename T>
tmd_status scan_inclusive(T *data, int64_t n, int64_t **tmp, int64_t *cap_tmp, cudaStream_t s,
                          int64_t level_start = 0) {
    // in-place inclusive scan; block sums of each recursion level live in the
    // int64 scratch at level_start (one int64 slot per block, T fits in it)
    if (n <= 0) return TMD_OK;
    const int64_t nb = (n + 2047) / 2048;
    if (nb == 1) {
        TMD_LAUNCH("k_scan_block", s, k_scan_block<T><<<1, 1024, 0, s>>>(data, n, nullptr));
        return TMD_OK;
    }
    if (level_start == 0) {
        int64_t need = 0, l = nb;
        while (l > 1) { need += l + 8; l = (l + 2047) / 2048; }
        tmd_status st = grow(tmp, cap_tmp, need + 64);
        if (st != TMD_OK) return st;
    }
    T *sums = reinterpret_cast<T *>(*tmp + level_start);
    TMD_LAUNCH("k_scan_block", s, k_scan_block<T><<<(unsigned)nb, 1024, 0, s>>>(data, n, sums));
    tmd_status st = scan_inclusive<T>(sums, nb, tmp, cap_tmp, s, level_start + nb + 8);
    if (st != TMD_OK) return st;
    TMD_LAUNCH("k_scan_add", s, k_scan_add<T><<<(unsigned)(nb - 1), 256, 0, s>>>(data, n, sums));
    return TMD_OK;
}

}  // namespace

void nlist_free(tmd_nlist *nl) {
    void *ptrs[] = {nl->cell_of, nl->cell_atoms, nl->cell_pos, nl->perm, nl->beg, nl->end, nl->counter, nl->sp, nl->cell_sys, nl->todo, nl->todo_count, nl->cell_start, nl->cell_fill, nl->nbr, nl->shift, nl->status, nl->type_block,
                    nl->type_start, nl->scan_tmp, nl->G, nl->dG, nl->P, nl->Fq, nl->part, nl->ph, nl->pl,
                    nl->io_pos, nl->io_types, nl->io_forces, nl->io_red, nl->pq, nl->pq2, nl->npair,
                    nl->perm_own, nl->own_count};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (nl->h_pinned) cudaFreeHost(nl->h_pinned);
    *nl = tmd_nlist();
}

tmd_status make_sys_params(const double box[3], const int32_t pbc[3], double r_list, SysParams *q, int64_t *ncell) {
    if (!(std::isfinite(r_list) && r_list > 0.0)) {
        set_error("r_list must be finite and > 0");
        return TMD_ERR_INVALID_ARG;
    }
    double Lmax = 0.0;
    int smax = 0;
    int64_t nct = 1;
    for (int x = 0; x < 3; ++x) {
        if (!(std::isfinite(box[x]) && box[x] > 0.0)) {
            set_error("box[%d] must be finite and > 0", x);
            return TMD_ERR_INVALID_ARG;
        }
        // cells are at least r_list + margin wide: the margin covers the
        // rounding of the cell assignment (an atom a hair inside a cell
        // boundary may be binned on either side of it)
        const double margin = 1e-6 + 1e-9 * box[x];
        int nc = (int)std::floor(box[x] / (r_list + margin));
        if (nc < 1) nc = 1;
        if (nc > 1024) nc = 1024;
        const double cs = box[x] / nc;
        int R = (int)std::ceil((r_list + margin) / cs);
        if (R < 1) R = 1;
        q->nc[x] = nc;
        q->R[x] = R;
        q->pbc[x] = pbc[x] ? 1 : 0;
        q->L[x] = box[x];
        q->ic[x] = nc / box[x];
        q->Lh[x] = (float)box[x];
        q->Ll[x] = (float)(box[x] - (double)q->Lh[x]);
        grid_split(box[x], q->Gh[x], q->Gl[x]);
        if (pbc[x]) {
            const int lo = -((R + nc - 1) / nc), hi = (nc - 1 + R) / nc;
            smax = std::max(smax, std::max(-lo, hi));
        }
        Lmax = std::max(Lmax, box[x]);
        nct *= nc;
    }
    if (smax > 15) {
        set_error("r_list %.3f needs image shifts beyond +-15 boxes", r_list);
        return TMD_ERR_CAPACITY;
    }
    if ((1.0 + smax) * Lmax >= GRID_LIMIT / 2) {
        set_error("box length %.1f A with image shifts up to %d: the pair geometry needs (1 + |s|) L < %.0f A",
                  Lmax, smax, GRID_LIMIT / 2);
        return TMD_ERR_CAPACITY;
    }
    q->r2 = r_list * r_list;
    {
        // FP32 screen error bound: |x_f - x| <= L 2^-24 per coordinate, the
        // shift product/difference add (1 + 2|s|) L 2^-24, the final
        // difference r 2^-24; squared-distance error <= 2 sqrt(3) r e + 3 e^2
        // + rounding of the sum.  Doubled for safety.
        const double u = std::ldexp(1.0, -24);
        const double e = ((4.0 + 4.0 * smax) * Lmax + 2.0 * (r_list + 1.0)) * u;
        const double rr = r_list + 1.0;
        const double margin = 2.0 * (2.0 * std::sqrt(3.0) * rr * e + 3.0 * e * e + 4.0 * rr * rr * u);
        q->r2lo = std::nextafter((float)(q->r2 - margin), -INFINITY);
        q->r2hi = std::nextafter((float)(q->r2 + margin), INFINITY);
    }
    q->cell_off = 0;
    *ncell = nct;
    return TMD_OK;
}

tmd_status build_tables(const double *pos, const int32_t *types, int64_t n, int n_sys, const SysParams *sp_host,
                        const int32_t *sys_of, const uint8_t *active, const int64_t *n_of_sys, int64_t ncell_total,
                        tmd_nlist *nl, cudaStream_t s, bool device_only) {
    if (device_only && (!nl->built || nl->n != n || nl->ncell != ncell_total || nl->cap_nnz < 1)) {
        set_error("a device-only rebuild needs a table built before with the same atoms and cells");
        return TMD_ERR_INVALID_ARG;
    }
    if (n < 0 || n >= (int64_t(1) << 28)) {
        set_error("n = %lld outside [0, 2^28)", (long long)n);
        return TMD_ERR_INVALID_ARG;
    }
    if (n > 0 && (!pos || !types)) {
        set_error("pos/types must be device pointers");
        return TMD_ERR_INVALID_ARG;
    }
    if (ncell_total >= (int64_t(1) << 31)) {
        set_error("too many binning cells");
        return TMD_ERR_CAPACITY;
    }
    nl->ncell = ncell_total;
    nl->n = n;
    if (!device_only) nl->built = 0;
    tmd_status st;
    const int64_t nb_bin = (n + BIN_THREADS - 1) / BIN_THREADS;
    if ((st = grow(&nl->cell_of, &nl->cap_atoms, n)) != TMD_OK) return st;
    if ((st = grow(&nl->cell_atoms, &nl->cap_cell_atoms, n)) != TMD_OK) return st;
    if ((st = grow(&nl->cell_pos, &nl->cap_cell_pos, n)) != TMD_OK) return st;
    if ((st = grow(&nl->perm, &nl->cap_perm, n)) != TMD_OK) return st;
    if ((st = grow(&nl->beg, &nl->cap_beg, n)) != TMD_OK) return st;
    if ((st = grow(&nl->end, &nl->cap_end, n)) != TMD_OK) return st;
    if ((st = grow(&nl->cell_start, &nl->cap_cells, ncell_total + 1)) != TMD_OK) return st;
    if ((st = grow(&nl->cell_fill, &nl->cap_cell_fill, ncell_total)) != TMD_OK) return st;
    if ((st = grow(&nl->type_block, &nl->cap_type_blocks, (nb_bin + 1) * TB_STRIDE)) != TMD_OK) return st;
    if ((st = grow(&nl->status, &nl->cap_status, 4)) != TMD_OK) return st;
    if ((st = grow(&nl->type_start, &nl->cap_type_start, TMD_MAX_SPECIES + 1)) != TMD_OK) return st;
    if ((st = grow(&nl->counter, &nl->cap_counter, 1)) != TMD_OK) return st;
    if ((st = grow(&nl->sp, &nl->cap_sp, n_sys)) != TMD_OK) return st;
    if (!nl->h_pinned) TMD_CUDA(cudaMallocHost((void **)&nl->h_pinned, 16 * sizeof(int64_t)));
    // device_only: the parameters and the capacities are those of the build
    // before (same box, same atoms); nothing is read back here
    if (!device_only) TMD_CUDA(cudaMemcpyAsync(nl->sp, sp_host, sizeof(SysParams) * n_sys, cudaMemcpyHostToDevice, s));
    // capacity for the entries: the previous table's size, or the uniform
    // density estimate, with headroom; a build that overflows is rerun once
    // with the exact size
    if (!device_only) {
        double est = 0.0;
        for (int k = 0; k < n_sys; ++k) {
            const double nk = (double)(n_of_sys ? n_of_sys[k] : n);
            const double vol = sp_host[k].L[0] * sp_host[k].L[1] * sp_host[k].L[2];
            const double r = std::sqrt(sp_host[k].r2);
            est += nk * (nk / vol) * (4.0 / 3.0) * M_PI * r * r * r;
        }
        const int64_t want = (int64_t)std::max<double>(1.2 * est, 1.1 * (double)nl->nnz) + 1024;
        if (nl->cap_nnz < want)
            if ((st = grow(&nl->nbr, &nl->cap_nnz, want)) != TMD_OK) return st;
        if (nl->cap_shift < nl->cap_nnz)
            if ((st = grow(&nl->shift, &nl->cap_shift, nl->cap_nnz)) != TMD_OK) return st;
    }
    TMD_CUDA(cudaMemsetAsync(nl->status, 0, sizeof(int32_t), s));
    TMD_CUDA(cudaMemsetAsync(nl->cell_start, 0, sizeof(int32_t) * (ncell_total + 1), s));
    TMD_CUDA(cudaMemsetAsync(nl->cell_fill, 0, sizeof(int32_t) * ncell_total, s));
    TMD_CUDA(cudaMemsetAsync(nl->type_start, 0, sizeof(int32_t) * (TMD_MAX_SPECIES + 1), s));
    TMD_CUDA(cudaMemsetAsync(nl->counter, 0, sizeof(unsigned long long), s));

    if (n > 0) {
        TMD_LAUNCH("k_bin", s, k_bin<<<(unsigned)nb_bin, BIN_THREADS, 0, s>>>(pos, types, n, nl->sp, sys_of, active,
                                                                            nl->cell_of, nl->cell_start,
                                                                            nl->type_block, nl->status));
        TMD_CUDA(cudaGetLastError());
        if ((st = scan_inclusive<int32_t>(nl->cell_start + 1, ncell_total, &nl->scan_tmp, &nl->cap_scan, s)) != TMD_OK)
            return st;
        TMD_LAUNCH("k_type_scan", s, k_type_scan<<<1, 128, 0, s>>>(nl->type_block, (int)nb_bin,
                                                                                    nl->type_start));
        TMD_LAUNCH("k_fill", s, k_fill<<<(unsigned)nb_bin, BIN_THREADS, 0, s>>>(pos, types, n, nl->cell_of, nl->cell_start,
                                                                              nl->cell_fill, nl->cell_atoms,
                                                                              nl->type_block, nl->type_start, nl->perm));
        const unsigned nb_cell = (unsigned)std::min<int64_t>((ncell_total + CELL_SORT_WARPS - 1) / CELL_SORT_WARPS, 65535);
        TMD_LAUNCH("k_cell_sort", s, k_cell_sort<<<nb_cell, CELL_SORT_WARPS * 32, 0, s>>>(
                                          nl->cell_start, ncell_total, nl->cell_atoms, pos, types, nl->cell_pos,
                                          nl->status));
        TMD_CUDA(cudaGetLastError());
    }

    const int32_t *cell_sys = nullptr;
    if (sys_of && n_sys > 1) {
        if ((st = grow(&nl->cell_sys, &nl->cap_cell_sys, ncell_total)) != TMD_OK) return st;
        dim3 g((unsigned)std::min<int64_t>(1024, 64), (unsigned)n_sys);
        TMD_LAUNCH("k_cell_sys", s, k_cell_sys<<<g, 256, 0, s>>>(nl->sp, n_sys, nl->cell_sys));
        cell_sys = nl->cell_sys;
    }
    if ((st = grow(&nl->todo, &nl->cap_todo, n + 1)) != TMD_OK) return st;
    if ((st = grow(&nl->todo_count, &nl->cap_todo_count, 1)) != TMD_OK) return st;

    NbrParams p;
    p.todo = nullptr;
    p.pos = pos;
    p.cell_of = nl->cell_of;
    p.cell_start = nl->cell_start;
    p.cell_pos = nl->cell_pos;
    p.sp = nl->sp;
    p.sys_of = sys_of;
    p.n = n;
    p.beg = nl->beg;
    p.end = nl->end;
    p.counter = nl->counter;
    p.status = nl->status;
    const size_t smem_atom = sizeof(uint64_t) * TMD_MAX_DEGREE * NBR_WARPS;
    const size_t smem_cell =
        sizeof(float4) * CAND_CAP + sizeof(char4) * CAND_CAP + sizeof(uint32_t) * 32 * (CAND_CAP / 32 + 1);
    static bool attr_set = false;
    if (!attr_set) {
        TMD_CUDA(cudaFuncSetAttribute(k_nbr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_atom));
        TMD_CUDA(cudaFuncSetAttribute(k_nbr_cell, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cell));
        attr_set = true;
    }
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const unsigned nb_cell = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ncell_total, (int64_t)std::max(nsm, 1) * 12));
    p.todo_n = nullptr;
    if (device_only) {
        // the cell pass, then the per-atom pass over a device-side count; the
        // caller checks the counter against the capacity and the status later
        p.nbr = nl->nbr;
        p.shift = nl->shift;
        p.cap = std::min(nl->cap_nnz, nl->cap_shift);
        TMD_CUDA(cudaMemsetAsync(nl->todo_count, 0, sizeof(unsigned long long), s));
        if (n > 0) {
            TMD_LAUNCH("k_nbr_cell", s, k_nbr_cell<<<nb_cell, CELL_WARPS * 32, smem_cell, s>>>(
                                            p, ncell_total, cell_sys, nl->cell_atoms, nl->todo, nl->todo_count));
            p.todo = nl->todo;
            p.todo_n = nl->todo_count;
            const unsigned gt = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + NBR_WARPS - 1) / NBR_WARPS,
                                                                                 (int64_t)std::max(nsm, 1) * 2));
            TMD_LAUNCH("k_nbr", s, k_nbr<<<gt, NBR_WARPS * 32, smem_atom, s>>>(p));
            TMD_CUDA(cudaGetLastError());
        }
        return TMD_OK;
    }
    int64_t nnz = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        p.nbr = nl->nbr;
        p.shift = nl->shift;
        p.cap = std::min(nl->cap_nnz, nl->cap_shift);
        p.todo = nullptr;
        p.n = n;
        TMD_CUDA(cudaMemsetAsync(nl->todo_count, 0, sizeof(unsigned long long), s));
        if (n > 0) {
            TMD_LAUNCH("k_nbr_cell", s, k_nbr_cell<<<nb_cell, CELL_WARPS * 32, smem_cell, s>>>(
                                            p, ncell_total, cell_sys, nl->cell_atoms, nl->todo, nl->todo_count));
            TMD_CUDA(cudaGetLastError());
        }
        TMD_CUDA(cudaMemcpyAsync(&nl->h_pinned[0], nl->counter, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        TMD_CUDA(cudaMemcpyAsync(&nl->h_pinned[1], nl->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        TMD_CUDA(cudaMemcpyAsync(&nl->h_pinned[2], nl->type_start, sizeof(int32_t) * (TMD_MAX_SPECIES + 1),
                                 cudaMemcpyDeviceToHost, s));
        TMD_CUDA(cudaMemcpyAsync(&nl->h_pinned[6], nl->todo_count, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        TMD_CUDA(cudaStreamSynchronize(s));
        const int64_t ntodo = nl->h_pinned[6];
        if (ntodo > 0) {  // atoms of cells with oversized stencils: per-atom pass
            p.todo = nl->todo;
            p.n = ntodo;
            TMD_LAUNCH("k_nbr", s, k_nbr<<<(unsigned)((ntodo + NBR_WARPS - 1) / NBR_WARPS), NBR_WARPS * 32, smem_atom, s>>>(p));
            TMD_CUDA(cudaGetLastError());
            TMD_CUDA(cudaMemcpyAsync(&nl->h_pinned[0], nl->counter, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            TMD_CUDA(cudaMemcpyAsync(&nl->h_pinned[1], nl->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            TMD_CUDA(cudaStreamSynchronize(s));
        }
        nnz = nl->h_pinned[0];
        int32_t status = 0;
        std::memcpy(&status, &nl->h_pinned[1], sizeof(int32_t));
        if (status & DEV_ERR_OUTSIDE_BOX) {
            set_error("an atom lies outside [0, L) on some axis (wrap periodic axes first)");
            return TMD_ERR_INVALID_ARG;
        }
        if (status & DEV_ERR_BAD_TYPE) {
            set_error("a species id is outside [0, %d)", TMD_MAX_SPECIES);
            return TMD_ERR_INVALID_ARG;
        }
        if (status & DEV_ERR_CELL) {
            set_error("a binning cell holds more than %d atoms", MAX_CELL);
            return TMD_ERR_CAPACITY;
        }
        if (status & DEV_ERR_DEGREE) {
            set_error("an atom has more than %d neighbour entries inside r_list", TMD_MAX_DEGREE);
            return TMD_ERR_CAPACITY;
        }
        if (nnz <= std::min(nl->cap_nnz, nl->cap_shift)) break;
        // overflow: nothing past the capacity was written; grow to the exact
        // size and build again
        if ((st = grow(&nl->nbr, &nl->cap_nnz, nnz)) != TMD_OK) return st;
        if ((st = grow(&nl->shift, &nl->cap_shift, nl->cap_nnz)) != TMD_OK) return st;
        TMD_CUDA(cudaMemsetAsync(nl->counter, 0, sizeof(unsigned long long), s));
    }
    int32_t tstart[TMD_MAX_SPECIES + 1];
    std::memcpy(tstart, &nl->h_pinned[2], sizeof(tstart));
    for (int t = 0; t < TMD_MAX_SPECIES; ++t) nl->type_count[t] = tstart[t + 1] - tstart[t];
    nl->n_active = tstart[TMD_MAX_SPECIES];
    nl->nnz = nnz;
    nl->built = 1;
    return TMD_OK;
}

tmd_status build_neighbors(const double *pos, const int32_t *types, int64_t n, const double box[3],
                           const int32_t pbc[3], double r_list, tmd_nlist *nl, cudaStream_t s) {
    SysParams q;
    int64_t ncell = 0;
    tmd_status st = make_sys_params(box, pbc, r_list, &q, &ncell);
    if (st != TMD_OK) return st;
    for (int x = 0; x < 3; ++x) {
        nl->nc[x] = q.nc[x];
        nl->R[x] = q.R[x];
        nl->pbc[x] = q.pbc[x];
        nl->box[x] = box[x];
    }
    nl->r_list = r_list;
    return build_tables(pos, types, n, 1, &q, nullptr, nullptr, nullptr, ncell, nl, s);
}

}  // namespace tmd
