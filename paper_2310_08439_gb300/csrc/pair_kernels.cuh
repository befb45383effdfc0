// Pair kernels of the TensorMD evaluation (Sec. "The Tensor Formalism"):
//   k_desc          setup (D, R, Dhat), H_abck = f_k f_c, M_abcd,
//                   P_abkd = sum_c H M, G_abkm = sigma(T_dm P^2)
//                                        -- Eqs. tensor_formalism, sigma_function
//   k_force(_merged) P' = 2 T sigma' P G'; V = P' H and W = P' H' (so that
//                   F1 = U H' R' = W . M and F2 = V M' with M' formed on the
//                   fly); ScatterSum into forces, virial
//                                        -- Eqs. dP_abkd, U_abck, F1_abcx, F2_abcx
//
// One warp owns one centre atom.  The in-cutoff pairs of each atom come from
// the pair cache (filled by k_screen in screen.cu, read by both passes) or,
// without a cache, from screening the table in the pass itself, compacted
// through a per-warp shared-memory queue; either way every lane works on an
// in-cutoff pair.  Each lane computes H and M for one
// neighbour and stages them in shared memory; the warp then accumulates the
// per-atom P[b][k][d] outer products with each lane owning a (K/8 x 5) block
// of P in registers.  In k_force each lane owns one cached pair and reads the
// atom's P' from shared memory with broadcast loads.
//
// Templates over the radial channel count K and the species count S; each
// pair_k<K>.cu translation unit instantiates one K (compiled in parallel).
#pragma once

#include "tmd_internal.cuh"

namespace tmd {

namespace {

constexpr int PW = PAIR_WARPS;   // warps per block in the pair kernels
constexpr float PI_F = 3.14159265358979323846f;

// multiplicities T_d and ranks m(d) in the row order of Eq. T_dm:
// 1 | x y z | xx xy xz yy yz zz | xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz
__constant__ float c_T[NMOM] = {1, 1, 1, 1, 1, 2, 2, 1, 2, 1, 1, 3, 3, 3, 6, 3, 1, 3, 3, 1};

__device__ __forceinline__ void moments20(float x, float y, float z, float *M) {
    M[0] = 1.f;
    M[1] = x; M[2] = y; M[3] = z;
    M[4] = x * x; M[5] = x * y; M[6] = x * z; M[7] = y * y; M[8] = y * z; M[9] = z * z;
    M[10] = M[4] * x; M[11] = M[4] * y; M[12] = M[4] * z; M[13] = x * M[7]; M[14] = M[5] * z;
    M[15] = x * M[9]; M[16] = M[7] * y; M[17] = M[7] * z; M[18] = y * M[9]; M[19] = M[9] * z;
}

// 2^x and 1/sqrt(x) from the special-function unit (PTX ex2.approx /
// rsqrt.approx, relative error about 2^-22; flush-to-zero: a result below
// 2^-126 becomes 0, and no argument here is subnormal)
__device__ __forceinline__ float ex2_ftz(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// sin(pi t) and cos(pi t) for |t| <= 1/2 from their Taylor series in
// y = pi t (|y| <= pi/2): the sine through y^13 and the cosine through y^12
// leave truncation errors of at most 7e-10 and 7e-9.
__device__ __forceinline__ void sincospi_half(float t, float &sn, float &cs) {
    const float y = PI_F * t, u = y * y;
    float p = 1.f / 6227020800.f;
    p = fmaf(p, u, -1.f / 39916800.f);
    p = fmaf(p, u, 1.f / 362880.f);
    p = fmaf(p, u, -1.f / 5040.f);
    p = fmaf(p, u, 1.f / 120.f);
    p = fmaf(p, u, -1.f / 6.f);
    sn = fmaf(y * u, p, y);
    float q = 1.f / 479001600.f;
    q = fmaf(q, u, -1.f / 3628800.f);
    q = fmaf(q, u, 1.f / 40320.f);
    q = fmaf(q, u, -1.f / 720.f);
    q = fmaf(q, u, 1.f / 24.f);
    q = fmaf(q, u, -0.5f);
    cs = fmaf(u, q, 1.f);
}

// f_c = (cos(pi r / rc) + 1) / 2 and df_c/dr for r < rc, through t = r / rc - 1/2:
// cos(pi r / rc) = -sin(pi t), sin(pi r / rc) = cos(pi t).
__device__ __forceinline__ void cutoff_fn(float r, float inv_rc, float &fc, float &dfc) {
    float sn, cs;
    sincospi_half(fmaf(r, inv_rc, -0.5f), sn, cs);
    fc = 0.5f - 0.5f * sn;
    dfc = -0.5f * PI_F * inv_rc * cs;
}

// H_k = f_k f_c (and dH_k/dr when DERIV) for r < rc, two channels at a time
// on packed FP32x2 arithmetic (fma/add/mul .f32x2 issue two FP32 operations as
// one instruction, each rounded as its scalar form).  The model's table holds
// (mu_hi, mu_lo, eta log2 e, 2 eta) per channel; r = r_hi + r_lo so that
// t = r - mu keeps ~FP64 accuracy (the Gaussians are steep: dlnH/dr = -2 eta t
// amplifies any rounding of r).  rad2 = the channel pairs of one species pair,
// two float4 per pair (k, k+1): (-mu_hi, -mu_hi', -mu_lo, -mu_lo') and
// (-eta log2 e, -eta' log2 e, -2 eta, -2 eta'), written by stage_rad2.
__device__ __forceinline__ void stage_rad2(float4 *dst, const float4 *src, int n) {
    for (int t = threadIdx.x; t < n / 2; t += blockDim.x) {
        const float4 a = src[2 * t], b = src[2 * t + 1];
        dst[2 * t] = make_float4(-a.x, -b.x, -a.y, -b.y);
        dst[2 * t + 1] = make_float4(-a.z, -b.z, -a.w, -b.w);
    }
}

struct Radial2 {
    float2 H, dH;
};

template <bool DERIV>
__device__ __forceinline__ Radial2 radial2(const float4 *rad2, int k, float2 rh2, float2 rl2, float2 fc2, float2 dfc2) {
    const float4 A = rad2[k], B = rad2[k + 1];   // channel pair k / 2
    const float2 t = __fadd2_rn(__fadd2_rn(rh2, make_float2(A.x, A.y)), __fadd2_rn(rl2, make_float2(A.z, A.w)));
    const float2 a = __fmul2_rn(__fmul2_rn(make_float2(B.x, B.y), t), t);
    const float2 f = make_float2(ex2_ftz(a.x), ex2_ftz(a.y));
    Radial2 o;
    o.H = __fmul2_rn(f, fc2);
    if (DERIV) o.dH = __fmul2_rn(f, __ffma2_rn(__fmul2_rn(make_float2(B.z, B.w), t), fc2, dfc2));
    return o;
}

// Tabulated radial basis (Sec. "The H_abck tensor and Batch Rational 1D
// Interpolation": H and H' read from a table with the cutoff folded in).
// Interval g = [g/scale, (g+1)/scale) holds, per k, the coefficients
// (c0, c1, c2, c3) of the cubic Hermite polynomial in t = r scale - g through
// H and H' at both ends; H = c0 + t (c1 + t (c2 + t c3)) and
// H' = scale (c1 + t (2 c2 + 3 t c3)).  scale is a power of two, so r_hi scale
// and its integer part are exact and t carries r_lo.  tab = the intervals of
// this species pair, [interval][k] float4.
struct TabCell {
    const float4 *c;   // this pair's interval: K float4
    float t, t3;       // t and 3 t
};

__device__ __forceinline__ TabCell tab_cell(const float *tab, int K, float scale, float r_hi, float r_lo) {
    const float x = r_hi * scale;
    const float gf = floorf(x);
    const int g = __float_as_int(gf + 12582912.0f) - 0x4B400000;   // exact: 0 <= gf < 2^22
    TabCell c;
    c.c = reinterpret_cast<const float4 *>(tab) + (size_t)g * K;
    c.t = (x - gf) + r_lo * scale;
    c.t3 = 3.f * c.t;
    return c;
}

__device__ __forceinline__ void tab_eval(const TabCell &tc, int k, float scale, float &H, float &dH) {
    const float4 q = __ldg(tc.c + k);
    H = fmaf(tc.t, fmaf(tc.t, fmaf(tc.t, q.w, q.z), q.y), q.x);
    dH = scale * fmaf(tc.t, fmaf(tc.t3, q.w, 2.f * q.z), q.y);
}

// channels k0 .. k0 + KC - 1 of a table of K channels
template <int KC, bool DERIV>
__device__ __forceinline__ void radial_tab(const float *tab, int K, int k0, float scale, float r_hi, float r_lo,
                                           float *H, float *dH) {
    const TabCell tc = tab_cell(tab, K, scale, r_hi, r_lo);
#pragma unroll
    for (int k = 0; k < KC; ++k) {
        float h, d;
        tab_eval(tc, k0 + k, scale, h, d);
        H[k] = h;
        if (DERIV) dH[k] = d;
    }
}

// r = |D| as an unevaluated sum r_hi + r_lo from r^2 = r2_hi + r2_lo, and 1/r.
// r_hi = r2 y with y ~ 1/sqrt(r2_hi) (pairs never coincide, r2_hi >= ~1); r_lo is the Newton correction (exact
// residual by FMA), so r_hi + r_lo is accurate to ~1e-13 whatever the error of
// y; 1/r is y refined by one Newton step against r_hi + r_lo.
__device__ __forceinline__ void split_sqrt(float r2_hi, float r2_lo, float &r_hi, float &r_lo, float &ir) {
    const float y = rsqrt_ftz(r2_hi);
    r_hi = r2_hi * y;
    r_lo = (fmaf(-r_hi, r_hi, r2_hi) + r2_lo) * 0.5f * y;
    const float e = fmaf(-r_hi, y, 1.f) - r_lo * y;
    ir = fmaf(y, e, y);
}

// Double-float helpers: a value is carried as an unevaluated sum hi + lo of two
// floats.  two_sum is Knuth's error-free addition.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// The box on the 2^-10 grid split: of the atom's system when batched
__device__ __forceinline__ void pair_box(const DevNlist &nl, int a, float (&Lh)[3], float (&Ll)[3]) {
    if (nl.sys_of) {
        const SysParams &q = nl.sp[nl.sys_of[a]];
#pragma unroll
        for (int x = 0; x < 3; ++x) { Lh[x] = q.Gh[x]; Ll[x] = q.Gl[x]; }
    } else {
#pragma unroll
        for (int x = 0; x < 3; ++x) { Lh[x] = nl.Lh[x]; Ll[x] = nl.Ll[x]; }
    }
}

// Pair geometry on the 2^-10 grid split (grid_split): every position and box
// length is hi + lo with hi a multiple of 2^-10 A and |lo| <= 2^-11 A.  Then
// D_hi = (x_j,hi - x_i,hi) + s L_hi is exact in FP32 (a multiple of 2^-10
// below 2^13 A in magnitude needs at most 23 significand bits; the box
// checks keep |s| L below 2^13), and D_lo = (x_j,lo - x_i,lo) + s L_lo is a
// small correction carried to ~1e-10 A.  |D|^2 is formed as an FP32 hi + lo
// pair from the exact squares of D_hi (FMA residuals, error-free sums) and the
// cross terms (2 D_hi + D_lo) D_lo, so r^2 keeps ~FP64 accuracy with no FP64
// instruction.  D itself is returned rounded to FP32.
__device__ __forceinline__ void pair_geom(const float4 jh, const float4 jl, const float4 ih, const float4 il,
                                          const char4 sh, const float (&Lh)[3], const float (&Ll)[3], float &dx,
                                          float &dy, float &dz, float &r2h, float &r2l) {
    // (float)s from the signed byte with one add and one subtract (|s| < 2^22)
    const float sx = __int_as_float(0x4B400000 + (int)sh.x) - 12582912.0f;
    const float sy = __int_as_float(0x4B400000 + (int)sh.y) - 12582912.0f;
    const float sz = __int_as_float(0x4B400000 + (int)sh.z) - 12582912.0f;
    const float hx = fmaf(sx, Lh[0], jh.x - ih.x), lx = fmaf(sx, Ll[0], jl.x - il.x);
    const float hy = fmaf(sy, Lh[1], jh.y - ih.y), ly = fmaf(sy, Ll[1], jl.y - il.y);
    const float hz = fmaf(sz, Lh[2], jh.z - ih.z), lz = fmaf(sz, Ll[2], jl.z - il.z);
    const float px = hx * hx, ex = fmaf(hx, hx, -px);
    const float py = hy * hy, ey = fmaf(hy, hy, -py);
    const float pz = hz * hz, ez = fmaf(hz, hz, -pz);
    float s1, e1, s2, e2;
    two_sum(px, py, s1, e1);
    two_sum(s1, pz, s2, e2);
    const float cross = fmaf(fmaf(2.f, hx, lx), lx, fmaf(fmaf(2.f, hy, ly), ly, fmaf(2.f, hz, lz) * lz));
    const float lo = ((ex + ey) + ez) + (e1 + e2) + cross;
    r2h = s2 + lo;
    r2l = lo - (r2h - s2);
    dx = hx + lx;
    dy = hy + ly;
    dz = hz + lz;
}

// Walk the entries [beg, end) of atom a, keep pairs with r^2 < rc^2 and hand
// them to f in batches of up to 32 (one per lane).  D = x_j + s L - x_i and r^2
// are formed in double-float FP32 arithmetic from hi/lo positions (no FP64
// instructions: on this GPU FP64 runs at a small fraction of the FP32 rate).
// The queue holds (Dx, Dy, Dz, j | b<<28) rounded to FP32 and r^2 as hi/lo.
// Used when there is no pair cache (k_screen in screen.cu fills the cache
// with the same pairs, in the same order, by the same arithmetic).
template <typename F>
__device__ __forceinline__ int for_pairs(const DevNlist &nl, int a, int64_t beg, int64_t end, float rc2h, float rc2l,
                                         float4 *q, float2 *q2, int lane, F &&f) {
    int qn = 0, kept = 0;
    const unsigned lt = (1u << lane) - 1u;
    const float4 ih = nl.ph[a], il = nl.pl[a];
    float Lh[3], Ll[3];
    pair_box(nl, a, Lh, Ll);
    int64_t base = beg;
    while (true) {
        while (qn < 32 && base < end) {
            const int64_t c = base + lane;
            bool v = false;
            float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
            float2 e2 = make_float2(0.f, 0.f);
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
            if (v) {
                const int slot = qn + __popc(m & lt);
                q[slot] = e;
                q2[slot] = e2;
            }
            qn += __popc(m);
            kept += __popc(m);
            base += 32;
        }
        if (qn == 0) break;
        // one call site: full batches while entries remain, then the tail
        const int nb = min(qn, 32);
        __syncwarp();
        f(q[lane], q2[lane], lane < nb, nb);
        __syncwarp();
        if (lane < qn - nb) {
            q[lane] = q[lane + 32];
            q2[lane] = q2[lane + 32];
        }
        __syncwarp();
        qn -= nb;
    }
    return kept;
}

// The in-cutoff pairs of atom a from the pair cache written by k_screen, in
// batches of up to 32 (one per lane).
template <typename F>
__device__ __forceinline__ void cached_pairs(const DevNlist &nl, int a, int np, int lane, F &&f) {
    const int64_t pb = nl.beg[a];
    for (int base = 0; base < np; base += 32) {
        const int nb = min(32, np - base);
        float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 e2 = make_float2(1.f, 0.f);
        if (lane < nb) {
            e = nl.pq[pb + base + lane];
            e2 = nl.pq2[pb + base + lane];
        }
        f(e, e2, lane < nb, nb);
    }
}

// A warp's stream of pair-cache batches over its atoms p, p + total, ...
// (perm order), read one batch ahead.
struct PairStream {
    int a = -1, np = 0;          // current atom and its in-cutoff pair count
    int64_t pb = 0;
    int an = -1, npn = 0;        // next atom (segment start and count read one atom ahead)
    int64_t pbn = 0;
    int an2 = -1;                // the atom after next (perm entry read two atoms ahead)
    float4 pf = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 pf2 = make_float2(1.f, 0.f);

    __device__ __forceinline__ void load(const DevNlist &nl, int64_t at, bool ok) {
        pf = make_float4(0.f, 0.f, 0.f, 0.f);
        pf2 = make_float2(1.f, 0.f);
        if (ok) {
            pf = nl.pq[at];
            pf2 = nl.pq2[at];
        }
    }
    __device__ __forceinline__ void start(const DevNlist &nl, int64_t p, int64_t total, int lane) {
        if (p < nl.n) {
            a = nl.perm[p];
            pb = nl.beg[a];
            np = nl.npair[a];
            load(nl, pb + lane, lane < np);
        }
        an = p + total < nl.n ? nl.perm[p + total] : -1;
    }
    // at the start of atom p: the next atom's segment, the perm entry after it
    __device__ __forceinline__ void atom_begins(const DevNlist &nl, int64_t p, int64_t total) {
        if (an >= 0) {
            pbn = nl.beg[an];
            npn = nl.npair[an];
        }
        an2 = p + 2 * total < nl.n ? nl.perm[p + 2 * total] : -1;
    }
    // the batch after the one starting at base: the atom's next batch, its
    // first batch again (another channel chunk follows), or the next atom's first
    __device__ __forceinline__ void advance(const DevNlist &nl, int base, bool again, int lane) {
        if (base + 32 < np)
            load(nl, pb + base + 32 + lane, lane < np - base - 32);
        else if (again)
            load(nl, pb + lane, lane < np);
        else
            load(nl, pbn + lane, an >= 0 && lane < npn);
    }
    __device__ __forceinline__ void atom_ends() {
        a = an;
        pb = pbn;
        np = an >= 0 ? npn : 0;
        an = an2;
    }
};

// ---------------------------------------------------------------------------
// descriptor forward: P and G per atom
// ---------------------------------------------------------------------------
// CACHED: the atom's in-cutoff pairs come from the pair cache filled by
// k_screen; otherwise the pass screens the table itself (for_pairs).  K > 32
// runs in chunks of 32 channels, each chunk going over the atom's pairs again,
// so that the per-lane accumulators and the staged columns stay those of
// K = 32.
template <int K, int S, bool TAB, bool CACHED>
__global__ void __launch_bounds__(PW * 32) k_desc(DevModel m, DevNlist nl, const double *__restrict__ pos,
                                                  const int32_t *__restrict__ types, float *__restrict__ G,
                                                  float *__restrict__ Pout) {
    constexpr int KC = K > 32 ? 32 : K;   // channels per chunk
    constexpr int KPL = KC / 8;           // k values per lane
    constexpr int RS = 44;       // row stride of the staged pair columns (>= 32 + 3 (S - 1) slots)
    constexpr int Dd = S * K * 4;
    __shared__ float4 s_rad2[S * S * K];
    __shared__ float4 s_q[PW][64];
    __shared__ float2 s_q2[PW][64];
    // staged pair data, one column per pair: H_k in row (k % KPL) 8 + k / KPL,
    // M_d in row (d % 5) 4 + d / 5, so that the lane owning k-group kg and
    // d-group g reads four pairs of a row with one conflict-free vector load
    __shared__ __align__(16) float s_H[PW][KC * RS];
    __shared__ __align__(16) float s_M[PW][NMOM * RS];
    stage_rad2(s_rad2, m.radial, S * S * K);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kg = lane >> 2, g = lane & 3;
    const unsigned lt = (1u << lane) - 1u;
    float Tg[5];
#pragma unroll
    for (int dd = 0; dd < 5; ++dd) Tg[dd] = c_T[5 * g + dd];
    const int64_t total = (int64_t)gridDim.x * PW;
    // CACHED: the pair-cache batches are read one batch ahead, across chunk
    // and atom boundaries (the next atom's segment one atom ahead, its perm
    // entry two atoms ahead), so that the pass waits on no load of its own
    // stream.  pf / pf2 hold the batch the next pair_fn call takes.
    PairStream ps;
    if constexpr (CACHED) ps.start(nl, (int64_t)blockIdx.x * PW + warp, total, lane);
    for (int64_t p = (int64_t)blockIdx.x * PW + warp; p < nl.n; p += total) {
        const int a = CACHED ? ps.a : nl.perm[p];
        const int ti = types[a];
        if constexpr (CACHED) ps.atom_begins(nl, p, total);
        for (int k0 = 0; k0 < K; k0 += KC) {
        // two partial sums per P entry (even and odd pair slots), so that
        // the accumulation runs on packed FP32x2 multiply-adds
        float2 acc2[S][KPL][5];
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int kk = 0; kk < KPL; ++kk)
#pragma unroll
                for (int dd = 0; dd < 5; ++dd) acc2[s][kk][dd] = make_float2(0.f, 0.f);
        float *sH = s_H[warp];
        float *sM = s_M[warp];
        auto pair_fn = [&](const float4 e, const float2 e2, bool valid, int) {
                      const uint32_t jb = __float_as_uint(e.w);
                      const int b = valid ? (int)(jb >> 28) : S;
                      // columns grouped by neighbour species, each group starting
                      // on a multiple of 4
                      int cnt[S], slot = 0, start = 0;
#pragma unroll
                      for (int s = 0; s < S; ++s) {
                          const unsigned ms = __ballot_sync(0xffffffffu, b == s);
                          if (b == s) slot = start + __popc(ms & lt);
                          cnt[s] = __popc(ms);
                          start += (cnt[s] + 3) & ~3;
                      }
                      if (valid) {
                          float r_hi, r_lo, ir;
                          split_sqrt(e2.x, e2.y, r_hi, r_lo, ir);
                          float H[KC], M[NMOM];
                          if (TAB)
                              radial_tab<KC, false>(m.rtab + (size_t)(ti * S + b) * m.rtab_n * 4 * K, K, k0,
                                                    m.rtab_scale, r_hi, r_lo, H, nullptr);
                          else {
                              float fc, dfc;
                              cutoff_fn(r_hi, m.inv_rc, fc, dfc);
                              const float4 *rad2 = &s_rad2[(ti * S + b) * K + k0];
#pragma unroll
                              for (int k = 0; k < KC; k += 2) {
                                  const Radial2 o = radial2<false>(rad2, k, make_float2(r_hi, r_hi),
                                                                   make_float2(r_lo, r_lo), make_float2(fc, fc),
                                                                   make_float2(dfc, dfc));
                                  H[k] = o.H.x;
                                  H[k + 1] = o.H.y;
                              }
                          }
                          moments20(e.x * ir, e.y * ir, e.z * ir, M);
#pragma unroll
                          for (int k = 0; k < KC; ++k) sH[((k % KPL) * 8 + k / KPL) * RS + slot] = H[k];
#pragma unroll
                          for (int d = 0; d < NMOM; ++d) sM[((d % 5) * 4 + d / 5) * RS + slot] = M[d];
                      }
                      __syncwarp();
                      // P[b][k][d] += H_k M_d: four pairs per step, the rest one at a time
                      start = 0;
#pragma unroll
                      for (int s = 0; s < S; ++s) {
                          const int stop = start + cnt[s];
                          int q = start;
                          for (; q + 4 <= stop; q += 4) {
                              float4 hv[KPL], mv[5];
#pragma unroll
                              for (int kk = 0; kk < KPL; ++kk)
                                  hv[kk] = *reinterpret_cast<const float4 *>(&sH[(kk * 8 + kg) * RS + q]);
#pragma unroll
                              for (int dd = 0; dd < 5; ++dd)
                                  mv[dd] = *reinterpret_cast<const float4 *>(&sM[(dd * 4 + g) * RS + q]);
#pragma unroll
                              for (int kk = 0; kk < KPL; ++kk)
#pragma unroll
                                  for (int dd = 0; dd < 5; ++dd) {
                                      float2 x = acc2[s][kk][dd];
                                      x = __ffma2_rn(make_float2(hv[kk].x, hv[kk].y), make_float2(mv[dd].x, mv[dd].y), x);
                                      x = __ffma2_rn(make_float2(hv[kk].z, hv[kk].w), make_float2(mv[dd].z, mv[dd].w), x);
                                      acc2[s][kk][dd] = x;
                                  }
                          }
                          for (; q < stop; ++q) {
                              float hv[KPL], mv[5];
#pragma unroll
                              for (int kk = 0; kk < KPL; ++kk) hv[kk] = sH[(kk * 8 + kg) * RS + q];
#pragma unroll
                              for (int dd = 0; dd < 5; ++dd) mv[dd] = sM[(dd * 4 + g) * RS + q];
#pragma unroll
                              for (int kk = 0; kk < KPL; ++kk)
#pragma unroll
                                  for (int dd = 0; dd < 5; ++dd)
                                      acc2[s][kk][dd].x = fmaf(hv[kk], mv[dd], acc2[s][kk][dd].x);
                          }
                          start += (cnt[s] + 3) & ~3;
                      }
                      __syncwarp();
                  };
        if constexpr (CACHED) {
            for (int base = 0; base < ps.np; base += 32) {
                const float4 e = ps.pf;
                const float2 e2 = ps.pf2;
                const int nb = min(32, ps.np - base);
                ps.advance(nl, base, k0 + KC < K, lane);
                pair_fn(e, e2, lane < nb, nb);
            }
            if (ps.np == 0 && k0 + KC >= K) ps.advance(nl, 0, false, lane);
        } else {
            for_pairs(nl, a, nl.beg[a], nl.end[a], m.rc2h, m.rc2l, s_q[warp], s_q2[warp], lane, pair_fn);
        }
        float acc[S][KPL][5];
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int kk = 0; kk < KPL; ++kk)
#pragma unroll
                for (int dd = 0; dd < 5; ++dd) acc[s][kk][dd] = acc2[s][kk][dd].x + acc2[s][kk][dd].y;
        // P[b][k][d] for the backward pass
        float *Pa = Pout + (size_t)p * (S * K * NMOM);   // workspaces are indexed by perm position
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int kk = 0; kk < KPL; ++kk)
#pragma unroll
                for (int dd = 0; dd < 5; ++dd)
                    Pa[(s * K + k0 + kg * KPL + kk) * NMOM + 5 * g + dd] = acc[s][kk][dd];
        // G[b][k][m] = sigma(sum_{d in rank m} T_d P^2)
#pragma unroll
        for (int s = 0; s < S; ++s) {
#pragma unroll
            for (int kk = 0; kk < KPL; ++kk) {
                float sq[5];
#pragma unroll
                for (int dd = 0; dd < 5; ++dd) sq[dd] = Tg[dd] * acc[s][kk][dd] * acc[s][kk][dd];
                const float tot = sq[0] + sq[1] + sq[2] + sq[3] + sq[4];
                // rank m of the four lanes g = 0..3 of this k: lane 0 holds
                // d = 0 (m = 0), d = 1..3 (m = 1) and d = 4 (m = 2); lane 1
                // d = 5..9 (m = 2); lanes 2 and 3 d = 10..19 (m = 3).  Lane g
                // writes G for m = g: m = 2 and m = 3 are pair sums (xor 1),
                // and lanes 1 and 2 fetch theirs from lane 0.
                const float s123 = sq[1] + sq[2] + sq[3];
                const float a = (g == 0) ? sq[4] : tot;
                const float asum = a + __shfl_xor_sync(0xffffffffu, a, 1);    // lanes 0, 1: m = 2; lanes 2, 3: m = 3
                const float m1 = __shfl_xor_sync(0xffffffffu, s123, 1);      // lane 1: lane 0's d = 1..3
                const float m2 = __shfl_xor_sync(0xffffffffu, asum, 2);      // lane 2: lane 0's m = 2
                // m = 0: sqrt(T_0 P^2) = |P| (T_0 = 1), taken as |P| so that a
                // channel's tiny P (|P| < 1e-19, whose square underflows in
                // FP32) is not read as 0; elsewhere bitwise the same value
                const float val = (g == 0) ? fabsf(acc[s][kk][0]) : ((g == 1) ? m1 : ((g == 2) ? m2 : asum));
                G[(size_t)p * Dd + (s * K + k0 + kg * KPL + kk) * 4 + g] = val;
            }
        }
        }
        if constexpr (CACHED) ps.atom_ends();
    }
}

// ---------------------------------------------------------------------------
// backward: P', pair gradients, ScatterSum, virial
// ---------------------------------------------------------------------------
// round(g * 2^32) as int64 (the 2^-32 fixed point of the ScatterSum) from
// 32-bit conversions only (on this GPU float <-> int64 conversions issue on
// the slow FP64 pipe); valid for |g| < 2^21.
__device__ __forceinline__ long long to_fixed(float g) {
    // two 32-bit stages: x = g 2^10 = r + v with r = rint(x) (|r| < 2^31 for
    // |g| < 2^21) and |v| <= 1/2 exact; then round(v 2^22) (exact scaling,
    // |.| <= 2^21): round(g 2^32) = r 2^22 + round(v 2^22), both roundings to
    // nearest even as a single rounding of g 2^32 would be
    const float x = g * 1024.0f;
    const float r = rintf(x);
    const int h1 = __float2int_rz(r);              // exact: r is an integer
    const int h2 = __float2int_rn((x - r) * 4194304.0f);
    return (long long)h1 * 4194304LL + (long long)h2;
}

// Sum of a fixed-point value over the 32 lanes of a warp, exact modulo 2^64
// (two's complement): each lane's value is cut into 21-, 21- and 22-bit
// chunks, whose lane sums (< 2^27) fit the 32-bit warp reduction, and the
// three sums are put back together.  Every lane receives the total.
__device__ __forceinline__ long long warp_sum_fixed(long long v) {
    const unsigned long long u = (unsigned long long)v;
    const unsigned c0 = __reduce_add_sync(0xffffffffu, (unsigned)(u & 0x1FFFFFull));
    const unsigned c1 = __reduce_add_sync(0xffffffffu, (unsigned)((u >> 21) & 0x1FFFFFull));
    const unsigned c2 = __reduce_add_sync(0xffffffffu, (unsigned)(u >> 42));
    return (long long)((unsigned long long)c0 + ((unsigned long long)c1 << 21) + ((unsigned long long)c2 << 42));
}

__device__ __forceinline__ void kahan_add(float &sum, float &comp, float x) {
    const float y = x - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

// The rest of g_ij once V_d and W_d of the pair are known, as packed pairs
// (d, d + 1).  The moments are formed in the same pairs, so that
// dE/dr = sum_d W_d M_d runs on FP32x2 multiply-adds.
__device__ __forceinline__ void pair_grad_tail(const float2 (&V2)[NMOM / 2], const float2 (&W2)[NMOM / 2], float ux,
                                               float uy, float uz, float ir, float &gxs, float &gys, float &gzs) {
    // M2[q] = (M_2q, M_2q+1) in the row order of moments20
    float2 M2[NMOM / 2];
    M2[0] = make_float2(1.f, ux);
    M2[1] = make_float2(uy, uz);
    M2[2] = make_float2(ux * ux, ux * uy);
    M2[3] = make_float2(ux * uz, uy * uy);
    M2[4] = make_float2(uy * uz, uz * uz);
    M2[5] = make_float2(M2[2].x * ux, M2[2].x * uy);
    M2[6] = make_float2(M2[2].x * uz, ux * M2[3].y);
    M2[7] = make_float2(M2[2].y * uz, ux * M2[4].y);
    M2[8] = make_float2(M2[3].y * uy, M2[3].y * uz);
    M2[9] = make_float2(uy * M2[4].y, M2[4].y * uz);
    float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < NMOM / 2; q += 2) {
        s0 = __ffma2_rn(W2[q], M2[q], s0);
        s1 = __ffma2_rn(W2[q + 1], M2[q + 1], s1);
    }
    const float dEdr = (s0.x + s0.y) + (s1.x + s1.y);
    // F2 = V M': dE/du_y = sum_d V_d dM_d/du_y (M' formed on the fly)
    const float xx = M2[2].x, xy = M2[2].y, xz = M2[3].x, yy = M2[3].y, yz = M2[4].x, zz = M2[4].y;
    auto V = [&](int d) { return (d & 1) ? V2[d >> 1].y : V2[d >> 1].x; };
    const float gx = V(1) + 2.f * ux * V(4) + uy * V(5) + uz * V(6) + 3.f * xx * V(10) +
                     2.f * xy * V(11) + 2.f * xz * V(12) + yy * V(13) + yz * V(14) + zz * V(15);
    const float gy = V(2) + ux * V(5) + 2.f * uy * V(7) + uz * V(8) + xx * V(11) + 2.f * xy * V(13) +
                     xz * V(14) + 3.f * yy * V(16) + 2.f * yz * V(17) + zz * V(18);
    const float gz = V(3) + ux * V(6) + uy * V(8) + 2.f * uz * V(9) + xx * V(12) + xy * V(14) +
                     2.f * xz * V(15) + yy * V(17) + 2.f * yz * V(18) + 3.f * zz * V(19);
    const float ug = ux * gx + uy * gy + uz * gz;
    // g_ij = dE/dD_ij = dE/dr u + (I - u u^T) dE/du / r
    gxs = fmaf(dEdr, ux, (gx - ux * ug) * ir);
    gys = fmaf(dEdr, uy, (gy - uy * ug) * ir);
    gzs = fmaf(dEdr, uz, (gz - uz * ug) * ir);
}

// g_ij = dE/dD_ij of one in-cutoff pair (Eqs. dP_abkd, U_abck, F1_abcx,
// F2_abcx): Pb = the centre atom's P' for the neighbour's species, rad = the
// radial parameters of the (centre, neighbour) species pair in the packed
// layout of stage_rad2.
template <int K, bool TAB>
__device__ __forceinline__ void pair_grad(const DevModel &m, const float4 e, const float2 e2, const float *Pb,
                                          const float4 *rad, const float *tab, float &gxs, float &gys, float &gzs) {
    float r_hi, r_lo, ir;
    split_sqrt(e2.x, e2.y, r_hi, r_lo, ir);
    const float ux = e.x * ir, uy = e.y * ir, uz = e.z * ir;
    // V_d = sum_k P'_kd H_k and W_d = sum_k P'_kd H'_k, so that
    // F1 = U H' R' = sum_d W_d M_d and F2 = V M'
    // V and W as packed pairs (d, d + 1): every multiply-add of the channel
    // loop is one FP32x2 instruction (each half rounded as fmaf)
    float2 V2[NMOM / 2], W2[NMOM / 2];
#pragma unroll
    for (int d = 0; d < NMOM / 2; ++d) V2[d] = W2[d] = make_float2(0.f, 0.f);
    float fc = 0.f, dfc = 0.f;
    TabCell tc;
    if (TAB)
        tc = tab_cell(tab, K, m.rtab_scale, r_hi, r_lo);
    else
        cutoff_fn(r_hi, m.inv_rc, fc, dfc);
    const float2 rh2 = make_float2(r_hi, r_hi), rl2 = make_float2(r_lo, r_lo);
    const float2 fc2 = make_float2(fc, fc), dfc2 = make_float2(dfc, dfc);
    constexpr int KU = K > 32 ? 16 : K;   // channels per unrolled block
#pragma unroll 1
    for (int kb = 0; kb < K; kb += KU)
#pragma unroll
    for (int ku = 0; ku < KU; ku += 2) {
        const int k = kb + ku;
        // H and H' of channels k, k + 1 formed inside the loop (no per-pair arrays)
        float Hk[2], dHk[2];
        if (TAB) {
            tab_eval(tc, k, m.rtab_scale, Hk[0], dHk[0]);
            tab_eval(tc, k + 1, m.rtab_scale, Hk[1], dHk[1]);
        } else {
            const Radial2 o = radial2<true>(rad, k, rh2, rl2, fc2, dfc2);
            Hk[0] = o.H.x; Hk[1] = o.H.y;
            dHk[0] = o.dH.x; dHk[1] = o.dH.y;
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const float2 h2 = make_float2(Hk[c], Hk[c]), d2 = make_float2(dHk[c], dHk[c]);
#pragma unroll
            for (int q4 = 0; q4 < NMOM / 4; ++q4) {
                const float4 pd = *reinterpret_cast<const float4 *>(Pb + (k + c) * NMOM + 4 * q4);
                const float2 plo = make_float2(pd.x, pd.y), phi = make_float2(pd.z, pd.w);
                V2[2 * q4] = __ffma2_rn(plo, h2, V2[2 * q4]);
                V2[2 * q4 + 1] = __ffma2_rn(phi, h2, V2[2 * q4 + 1]);
                W2[2 * q4] = __ffma2_rn(plo, d2, W2[2 * q4]);
                W2[2 * q4 + 1] = __ffma2_rn(phi, d2, W2[2 * q4 + 1]);
            }
        }
    }
    pair_grad_tail(V2, W2, ux, uy, uz, ir, gxs, gys, gzs);
}


// P'_bkd = 2 T_d sigma'_m P_bkd G'_bkm (for m = 0: G'_bk0 sign(P)) of the
// atom at perm position p (P and G' are indexed by perm position) into a
// shared slot, each lane its (K/8 x 5) block  (Eq. dP_abkd)
template <int K, int S>
__device__ __forceinline__ void pprime_setup(const float *__restrict__ Pin, const float *__restrict__ dG, int p,
                                             float *slot, int kg, int g, const float (&Tg)[5]) {
    constexpr int KPL = K / 8;
    constexpr int PSTR = K * NMOM + 4;
    constexpr int Dd = S * K * 4;
    const float *Pa = Pin + (size_t)p * (S * K * NMOM);
    const float *dGa = dG + (size_t)p * Dd;
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
        for (int kk = 0; kk < KPL; ++kk) {
            const int k = kg * KPL + kk;
            const float4 gm = *reinterpret_cast<const float4 *>(dGa + (s * K + k) * 4);
#pragma unroll
            for (int dd = 0; dd < 5; ++dd) {
                const int d = 5 * g + dd;
                const float pv = Pa[(s * K + k) * NMOM + d];
                float gg;
                if (g == 0) gg = (dd == 0) ? gm.x : ((dd < 4) ? gm.y : gm.z);
                else gg = (g == 1) ? gm.z : gm.w;
                float v;
                if (g == 0 && dd == 0) v = (pv > 0.f) ? gg : ((pv < 0.f) ? -gg : 0.f);
                else v = 2.f * Tg[dd] * pv * gg;
                slot[s * PSTR + k * NMOM + d] = v;
            }
        }
}

// Lane sums of the virial -> warp total (FP32, fixed butterfly order) added to
// the warp's FP64 accumulator; the lane sums restart from zero.  A lane sums
// the pairs of about VFLUSH / 32 of the warp's atoms between flushes, so the
// FP32 rounding stays at the level of one atom's virial.
constexpr int VFLUSH = 8;
__device__ __forceinline__ void virial_flush(float (&wacc)[9], double *acc, int lane) {
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        float v = wacc[t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) acc[t] += (double)v;
        wacc[t] = 0.f;
    }
}

// Force pass over the pair cache with full lane batches: each warp walks a
// contiguous run of atoms (perm order) and fills every batch of 32 lanes with
// the rest of the current atom's pairs followed by the first pairs of the
// next atom (two P' slots per warp, two self-force accumulators).
template <int K, int S, bool TAB>
__global__ void __launch_bounds__(PW * 32, 4) k_force_merged(DevModel m, DevNlist nl, const int32_t *__restrict__ types,
                                                          const float *__restrict__ Pin, const float *__restrict__ dG,
                                                          unsigned long long *__restrict__ Fq,
                                                          double *__restrict__ part_w) {
    constexpr int PSTR = K * NMOM + 4;
    __shared__ float4 s_rad[S * S * K];
    __shared__ __align__(16) float s_Pd[PW][2][S * PSTR];
    __shared__ double s_w[PW][9];
    stage_rad2(s_rad, m.radial, S * S * K);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane < 9) s_w[warp][lane] = 0.0;
    __syncthreads();
    const int kg = lane >> 2, g = lane & 3;
    float Tg[5];
#pragma unroll
    for (int dd = 0; dd < 5; ++dd) Tg[dd] = c_T[5 * g + dd];
    // virial: each lane's pairs summed in FP32 over VFLUSH atoms, then the
    // warp's total added to an FP64 accumulator in shared memory
    float wacc[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) wacc[t] = 0.f;
    int since = 0;
    const int64_t nw = (int64_t)gridDim.x * PW, wid = (int64_t)blockIdx.x * PW + warp;
    const int64_t chunk = (nl.n + nw - 1) / nw;
    int64_t p = wid * chunk;
    const int64_t pend = min(nl.n, p + chunk);
    if (p < pend) {
        int slot = 0;
        int a = nl.perm[p], ta = types[a];
        pprime_setup<K, S>(Pin, dG, (int)p, s_Pd[warp][0], kg, g, Tg);
        int64_t cb = nl.beg[a];
        int cr = nl.npair[a];
        long long fcx = 0, fcy = 0, fcz = 0;
        while (p < pend) {
            const int take_c = min(cr, 32);
            const bool has_n = cr < 32 && p + 1 < pend;
            int take_n = 0, an = 0, tn = 0, nr = 0;
            int64_t nb = 0;
            if (has_n) {   // bring in the next atom
                an = nl.perm[p + 1];
                tn = types[an];
                pprime_setup<K, S>(Pin, dG, (int)p + 1, s_Pd[warp][slot ^ 1], kg, g, Tg);
                nb = nl.beg[an];
                nr = nl.npair[an];
                take_n = min(nr, 32 - cr);
            }
            __syncwarp();
            long long fnx = 0, fny = 0, fnz = 0;
            const bool isc = lane < take_c, isn = !isc && lane < take_c + take_n;
            if (isc || isn) {
                const int64_t c = isc ? cb + lane : nb + (lane - take_c);
                const float4 e = nl.pq[c];
                const float2 e2 = nl.pq2[c];
                const uint32_t jb = __float_as_uint(e.w);
                const int b = (int)(jb >> 28);
                const int j = (int)(jb & 0x0FFFFFFFu);
                const float *Pb = s_Pd[warp][isc ? slot : slot ^ 1] + b * PSTR;
                const int tp = (isc ? ta : tn) * S + b;
                float gxs, gys, gzs;
                pair_grad<K, TAB>(m, e, e2, Pb, &s_rad[tp * K], TAB ? m.rtab + (size_t)tp * m.rtab_n * 4 * K : nullptr,
                                  gxs, gys, gzs);
                // ScatterSum in 2^-32 fixed point (exact, order independent)
                const long long qx = to_fixed(gxs);
                const long long qy = to_fixed(gys);
                const long long qz = to_fixed(gzs);
                if (isc) { fcx += qx; fcy += qy; fcz += qz; }
                else { fnx = qx; fny = qy; fnz = qz; }
                atomicAdd(&Fq[3 * (int64_t)j], (unsigned long long)(-qx));
                atomicAdd(&Fq[3 * (int64_t)j + 1], (unsigned long long)(-qy));
                atomicAdd(&Fq[3 * (int64_t)j + 2], (unsigned long long)(-qz));
                const float D[3] = {e.x, e.y, e.z};
                const float gv[3] = {gxs, gys, gzs};
#pragma unroll
                for (int al = 0; al < 3; ++al)
#pragma unroll
                    for (int be = 0; be < 3; ++be) wacc[al * 3 + be] = fmaf(-D[al], gv[be], wacc[al * 3 + be]);
            }
            cb += take_c;
            cr -= take_c;
            if (cr == 0) {   // the current atom is complete: its own force
                fcx = warp_sum_fixed(fcx);
                fcy = warp_sum_fixed(fcy);
                fcz = warp_sum_fixed(fcz);
                if (lane == 0) {
                    atomicAdd(&Fq[3 * (int64_t)a], (unsigned long long)fcx);
                    atomicAdd(&Fq[3 * (int64_t)a + 1], (unsigned long long)fcy);
                    atomicAdd(&Fq[3 * (int64_t)a + 2], (unsigned long long)fcz);
                }
                if (++since == VFLUSH) {
                    virial_flush(wacc, s_w[warp], lane);
                    since = 0;
                }
                ++p;
                if (p < pend) {
                    if (has_n) {   // the next atom (already set up) becomes the current one
                        a = an;
                        ta = tn;
                        slot ^= 1;
                        cb = nb + take_n;
                        cr = nr - take_n;
                        fcx = fnx; fcy = fny; fcz = fnz;
                    } else {
                        __syncwarp();
                        a = nl.perm[p];
                        ta = types[a];
                        pprime_setup<K, S>(Pin, dG, (int)p, s_Pd[warp][slot], kg, g, Tg);
                        cb = nl.beg[a];
                        cr = nl.npair[a];
                        fcx = fcy = fcz = 0;
                    }
                }
            }
            __syncwarp();
        }
    }
    virial_flush(wacc, s_w[warp], lane);
    __syncthreads();
    if (threadIdx.x < 9) {
        double v = 0.0;
        for (int w = 0; w < PW; ++w) v += s_w[w][threadIdx.x];
        part_w[(size_t)blockIdx.x * 9 + threadIdx.x] = v;
    }
}

// ---------------------------------------------------------------------------
// force pass with the per-atom contractions on tensor cores
// ---------------------------------------------------------------------------
// For one atom the pair sums V_jd = sum_k H_jk P'_kd and W_jd = sum_k H'_jk P'_kd
// (Eqs. U_abck, F1_abcx, F2_abcx) are one matrix product: [H; H'] (rows =
// pairs, columns = k) times P' (k x d).  Each warp takes its atom's cached
// pairs 32 at a time: every lane forms H and H' of its pair into a shared
// 64 x K tile (rows 0-31 H, rows 32-63 H'), the warp multiplies the tile by P'
// with mma.sync m16n8k8 on TF32 operands (d padded to 24 with zeros), and
// every lane reads back the V and W rows of its pair for the rest of g_ij.
// FP32 accuracy from TF32 products: each operand x is split into
// x_hi = tf32(x) and x_lo = tf32(x - x_hi), and a product is accumulated as
// a_lo b_hi + a_hi b_lo + a_hi b_hi in FP32 (the dropped a_lo b_lo and the
// split remainders are about 2^-22 of |a b|).
__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo) {
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(x));
    const float rest = x - __uint_as_float(hi);   // exact
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(rest));
}

// c += a b for one m16n8k8 tile (a: 16 x 8 row-major, b: 8 x 8, c: 16 x 8)
__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One species, direct radial basis, pair cache present.
template <int K>
__global__ void __launch_bounds__(PW * 32, 4) k_force_tc(DevModel m, DevNlist nl, const float *__restrict__ Pin,
                                                      const float *__restrict__ dG,
                                                      unsigned long long *__restrict__ Fq,
                                                      double *__restrict__ part_w) {
    static_assert(K % 8 == 0 && K <= 32, "k steps of 8, one pass");
    constexpr int KS = K / 8;        // k steps of the product
    constexpr int AS = K + 4;        // row stride of the H / H' tile (conflict-free fragment loads)
    constexpr int CS = 28;           // row stride of the V / W tile (24 columns, 16-byte rows)
    constexpr int PSTR = K * NMOM + 4;
    // the V / W tile is written over the H / H' tile, one m tile at a time,
    // in descending order when its rows are longer (CS > AS) and ascending
    // otherwise: the words a tile's results land on then hold only H / H'
    // rows of this tile (already in registers) or of tiles already multiplied
    constexpr int TILE = (64 * CS > 64 * AS) ? 64 * CS : 64 * AS;
    constexpr bool ASCENDING = AS >= CS;
    __shared__ float4 s_rad[K];
    __shared__ __align__(16) float s_Pd[PW][PSTR];
    __shared__ __align__(16) float s_T[PW][TILE];
    __shared__ double s_w[PW][9];
    for (int t = threadIdx.x; t < K; t += blockDim.x) s_rad[t] = m.radial[t];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kg = lane >> 2, g = lane & 3;   // P' setup block; also the fragment row / column group
    float Tg[5];
#pragma unroll
    for (int dd = 0; dd < 5; ++dd) Tg[dd] = c_T[5 * g + dd];
    float wsum[9], wcmp[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) { wsum[t] = 0.f; wcmp[t] = 0.f; }
    float *sPd = s_Pd[warp];
    float *sT = s_T[warp];
    const int64_t total = (int64_t)gridDim.x * PW;
    for (int64_t p = (int64_t)blockIdx.x * PW + warp; p < nl.n; p += total) {
        const int a = nl.perm[p];
        pprime_setup<K, 1>(Pin, dG, (int)p, sPd, kg, g, Tg);
        __syncwarp();
        // B fragments of P' (k x 24), hi and lo parts: b0 = (k = t, n = g), b1 = (k = t + 4, n = g)
        uint32_t bh[KS][3][2], bl[KS][3][2];
#pragma unroll
        for (int ks = 0; ks < KS; ++ks)
#pragma unroll
            for (int nt = 0; nt < 3; ++nt)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = ks * 8 + g + 4 * h, d = nt * 8 + kg;
                    split_tf32(d < NMOM ? sPd[k * NMOM + d] : 0.f, bh[ks][nt][h], bl[ks][nt][h]);
                }
        const int np = nl.npair[a];
        const int64_t pb = nl.beg[a];
        long long fx = 0, fy = 0, fz = 0;
        float wa[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) wa[t] = 0.f;
        for (int base = 0; base < np; base += 32) {
            const int nb = min(32, np - base);
            const bool valid = lane < nb;
            float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
            float2 e2 = make_float2(1.f, 0.f);
            if (valid) {
                e = nl.pq[pb + base + lane];
                e2 = nl.pq2[pb + base + lane];
            }
            float r_hi, r_lo, ir;
            split_sqrt(e2.x, e2.y, r_hi, r_lo, ir);
            {   // H and H' of this lane's pair into rows lane and 32 + lane (zeros for idle lanes)
                float fc, dfc;
                cutoff_fn(r_hi, m.inv_rc, fc, dfc);
                if (!valid) fc = dfc = 0.f;
                float *hrow = sT + lane * AS, *drow = sT + (32 + lane) * AS;
#pragma unroll
                for (int k4 = 0; k4 < K; k4 += 4) {
                    float hv[4], dv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float4 rp = s_rad[k4 + u];
                        const float t = (r_hi - rp.x) + (r_lo - rp.y);
                        const float f = ex2_ftz(-rp.z * t * t);
                        hv[u] = f * fc;
                        dv[u] = f * fmaf(-rp.w * t, fc, dfc);
                    }
                    *reinterpret_cast<float4 *>(hrow + k4) = make_float4(hv[0], hv[1], hv[2], hv[3]);
                    *reinterpret_cast<float4 *>(drow + k4) = make_float4(dv[0], dv[1], dv[2], dv[3]);
                }
            }
            __syncwarp();
            // [H; H'] P' -> V / W rows (m tiles 0, 1: H; 2, 3: H'); tiles past
            // the last pair are skipped
            const int mt_used = (nb + 15) >> 4;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int mt = ASCENDING ? i : 3 - i;
                if ((mt & 1) >= mt_used) continue;
                float c[3][4];
#pragma unroll
                for (int nt = 0; nt < 3; ++nt)
#pragma unroll
                    for (int q = 0; q < 4; ++q) c[nt][q] = 0.f;
#pragma unroll
                for (int ks = 0; ks < KS; ++ks) {
                    const float *r0 = sT + (mt * 16 + kg) * AS + ks * 8 + g;
                    const float *r1 = r0 + 8 * AS;
                    uint32_t ah[4], al[4];
                    split_tf32(r0[0], ah[0], al[0]);
                    split_tf32(r1[0], ah[1], al[1]);
                    split_tf32(r0[4], ah[2], al[2]);
                    split_tf32(r1[4], ah[3], al[3]);
#pragma unroll
                    for (int nt = 0; nt < 3; ++nt) {
                        mma_tf32(c[nt], al, bh[ks][nt][0], bh[ks][nt][1]);
                        mma_tf32(c[nt], ah, bl[ks][nt][0], bl[ks][nt][1]);
                        mma_tf32(c[nt], ah, bh[ks][nt][0], bh[ks][nt][1]);
                    }
                }
                __syncwarp();   // every lane's fragment loads of this tile precede the stores below
#pragma unroll
                for (int nt = 0; nt < 3; ++nt) {
                    float *c0 = sT + (mt * 16 + kg) * CS + nt * 8 + 2 * g;
                    *reinterpret_cast<float2 *>(c0) = make_float2(c[nt][0], c[nt][1]);
                    *reinterpret_cast<float2 *>(c0 + 8 * CS) = make_float2(c[nt][2], c[nt][3]);
                }
                __syncwarp();
            }
            if (valid) {
                float2 V2[NMOM / 2], W2[NMOM / 2];
                const float *vr = sT + lane * CS, *wr = sT + (32 + lane) * CS;
#pragma unroll
                for (int q4 = 0; q4 < NMOM / 4; ++q4) {
                    const float4 v = *reinterpret_cast<const float4 *>(vr + 4 * q4);
                    const float4 w = *reinterpret_cast<const float4 *>(wr + 4 * q4);
                    V2[2 * q4] = make_float2(v.x, v.y); V2[2 * q4 + 1] = make_float2(v.z, v.w);
                    W2[2 * q4] = make_float2(w.x, w.y); W2[2 * q4 + 1] = make_float2(w.z, w.w);
                }
                float gxs, gys, gzs;
                pair_grad_tail(V2, W2, e.x * ir, e.y * ir, e.z * ir, ir, gxs, gys, gzs);
                const int j = (int)(__float_as_uint(e.w) & 0x0FFFFFFFu);
                // ScatterSum in 2^-32 fixed point (exact, order independent)
                const long long qx = to_fixed(gxs);
                const long long qy = to_fixed(gys);
                const long long qz = to_fixed(gzs);
                fx += qx; fy += qy; fz += qz;
                atomicAdd(&Fq[3 * (int64_t)j], (unsigned long long)(-qx));
                atomicAdd(&Fq[3 * (int64_t)j + 1], (unsigned long long)(-qy));
                atomicAdd(&Fq[3 * (int64_t)j + 2], (unsigned long long)(-qz));
                const float D[3] = {e.x, e.y, e.z};
                const float gv[3] = {gxs, gys, gzs};
#pragma unroll
                for (int al = 0; al < 3; ++al)
#pragma unroll
                    for (int be = 0; be < 3; ++be) wa[al * 3 + be] = fmaf(-D[al], gv[be], wa[al * 3 + be]);
            }
            __syncwarp();   // the tile is rewritten by the next batch
        }
        fx = warp_sum_fixed(fx);
        fy = warp_sum_fixed(fy);
        fz = warp_sum_fixed(fz);
        if (lane == 0) {
            atomicAdd(&Fq[3 * (int64_t)a], (unsigned long long)fx);
            atomicAdd(&Fq[3 * (int64_t)a + 1], (unsigned long long)fy);
            atomicAdd(&Fq[3 * (int64_t)a + 2], (unsigned long long)fz);
        }
#pragma unroll
        for (int t = 0; t < 9; ++t) kahan_add(wsum[t], wcmp[t], wa[t]);
        __syncwarp();   // sPd is rewritten by the next atom
    }
    // virial: per-lane compensated sums -> warp total as an FP32 double-float -> FP64 block total
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        float hi = wsum[t], lo = -wcmp[t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
            float sh, se;
            two_sum(hi, oh, sh, se);
            lo = (lo + ol) + se;
            two_sum(sh, lo, hi, lo);
        }
        if (lane == 0) s_w[warp][t] = (double)hi + (double)lo;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        double v = 0.0;
        for (int w = 0; w < PW; ++w) v += s_w[w][threadIdx.x];
        part_w[(size_t)blockIdx.x * 9 + threadIdx.x] = v;
    }
}

// PAW (batched): each atom's virial is summed over its own pairs and written
// to w_atom [atoms][9] for per-system reductions; otherwise lanes keep
// compensated running sums and each block writes one FP64 partial.
template <int K, int S, bool PAW, bool CACHED, bool TAB>
__global__ void __launch_bounds__(PW * 32, 4) k_force(DevModel m, DevNlist nl, const double *__restrict__ pos,
                                                   const int32_t *__restrict__ types, const float *__restrict__ Pin,
                                                   const float *__restrict__ dG,
                                                   unsigned long long *__restrict__ Fq,
                                                   double *__restrict__ part_w, float *__restrict__ w_atom) {
    constexpr int KPL = K / 8;
    constexpr int PSTR = K * NMOM + 4;   // per-species stride of P' (bank offset between species)
    constexpr int Dd = S * K * 4;
    __shared__ float4 s_rad[S * S * K];
    __shared__ float4 s_q[PW][64];
    __shared__ float2 s_q2[PW][64];
    __shared__ __align__(16) float s_Pd[PW][S * PSTR];
    __shared__ double s_w[PW][9];
    stage_rad2(s_rad, m.radial, S * S * K);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kg = lane >> 2, g = lane & 3;
    float Tg[5];
#pragma unroll
    for (int dd = 0; dd < 5; ++dd) Tg[dd] = c_T[5 * g + dd];
    float wsum[9], wcmp[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) { wsum[t] = 0.f; wcmp[t] = 0.f; }
    float *sPd = s_Pd[warp];
    const int64_t total = (int64_t)gridDim.x * PW;
    for (int64_t p = (int64_t)blockIdx.x * PW + warp; p < nl.n; p += total) {
        const int a = nl.perm[p];
        const int ti = types[a];
        // P'_bkd = 2 T_d sigma'_m P_bkd G'_bkm; for m = 0: G'_bk0 sign(P)  (Eq. dP_abkd)
        const float *Pa = Pin + (size_t)p * (S * K * NMOM);
        const float *dGa = dG + (size_t)p * Dd;
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
            for (int kk = 0; kk < KPL; ++kk) {
                const int k = kg * KPL + kk;
                const float4 gm = *reinterpret_cast<const float4 *>(dGa + (s * K + k) * 4);
#pragma unroll
                for (int dd = 0; dd < 5; ++dd) {
                    const int d = 5 * g + dd;
                    const float pv = Pa[(s * K + k) * NMOM + d];
                    // rank of d: g==0 -> {0,1,1,1,2}, g==1 -> 2, g>=2 -> 3
                    float gg;
                    if (g == 0) gg = (dd == 0) ? gm.x : ((dd < 4) ? gm.y : gm.z);
                    else gg = (g == 1) ? gm.z : gm.w;
                    float v;
                    if (g == 0 && dd == 0) v = (pv > 0.f) ? gg : ((pv < 0.f) ? -gg : 0.f);
                    else v = 2.f * Tg[dd] * pv * gg;
                    sPd[s * PSTR + k * NMOM + d] = v;
                }
            }
        __syncwarp();
        long long fx = 0, fy = 0, fz = 0;
        float wa[9];  // this lane's pairs of this atom
#pragma unroll
        for (int t = 0; t < 9; ++t) wa[t] = 0.f;
        auto pair_fn = [&](const float4 e, const float2 e2, bool valid, int) {
                      if (!valid) return;
                      const uint32_t jb = __float_as_uint(e.w);
                      const int b = (int)(jb >> 28);
                      const int j = (int)(jb & 0x0FFFFFFFu);
                      float gxs, gys, gzs;
                      pair_grad<K, TAB>(m, e, e2, sPd + b * PSTR, &s_rad[(ti * S + b) * K],
                                        TAB ? m.rtab + (size_t)(ti * S + b) * m.rtab_n * 4 * K : nullptr, gxs, gys, gzs);
                      // ScatterSum in 2^-32 fixed point: integer adds are exact and
                      // order independent, so forces are bitwise reproducible.
                      const long long qx = to_fixed(gxs);
                      const long long qy = to_fixed(gys);
                      const long long qz = to_fixed(gzs);
                      fx += qx; fy += qy; fz += qz;
                      atomicAdd(&Fq[3 * (int64_t)j], (unsigned long long)(-qx));
                      atomicAdd(&Fq[3 * (int64_t)j + 1], (unsigned long long)(-qy));
                      atomicAdd(&Fq[3 * (int64_t)j + 2], (unsigned long long)(-qz));
                      const float D[3] = {e.x, e.y, e.z};
                      const float gv[3] = {gxs, gys, gzs};
#pragma unroll
                      for (int al = 0; al < 3; ++al)
#pragma unroll
                          for (int be = 0; be < 3; ++be) wa[al * 3 + be] = fmaf(-D[al], gv[be], wa[al * 3 + be]);
                  };
        if constexpr (CACHED)
            cached_pairs(nl, a, nl.npair[a], lane, pair_fn);
        else
            for_pairs(nl, a, nl.beg[a], nl.end[a], m.rc2h, m.rc2l, s_q[warp], s_q2[warp], lane, pair_fn);
        fx = warp_sum_fixed(fx);
        fy = warp_sum_fixed(fy);
        fz = warp_sum_fixed(fz);
        if (lane == 0) {
            atomicAdd(&Fq[3 * (int64_t)a], (unsigned long long)fx);
            atomicAdd(&Fq[3 * (int64_t)a + 1], (unsigned long long)fy);
            atomicAdd(&Fq[3 * (int64_t)a + 2], (unsigned long long)fz);
        }
        if constexpr (PAW) {
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                float v = wa[t];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) w_atom[(size_t)a * 9 + t] = v;
            }
        } else {
#pragma unroll
            for (int t = 0; t < 9; ++t) kahan_add(wsum[t], wcmp[t], wa[t]);
        }
        __syncwarp();
    }
    // virial: per-lane compensated sums (value = sum - comp) -> warp total as
    // an FP32 double-float (error-free additions) -> FP64 block total
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        float hi = wsum[t], lo = -wcmp[t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
            float sh, se;
            two_sum(hi, oh, sh, se);
            lo = (lo + ol) + se;
            two_sum(sh, lo, hi, lo);
        }
        if (lane == 0) s_w[warp][t] = (double)hi + (double)lo;
    }
    __syncthreads();
    if (!PAW && threadIdx.x < 9) {
        double v = 0.0;
        for (int w = 0; w < PW; ++w) v += s_w[w][threadIdx.x];
        part_w[(size_t)blockIdx.x * 9 + threadIdx.x] = v;
    }
}

template <int K, int S>
tmd_status launch_pair_kernels(const DevModel &dm, const DevNlist &dn, const double *pos, const int32_t *types,
                               tmd_nlist *nl, double *part_w, int nblk, cudaStream_t s, bool forward,
                               float *w_atom) {
    if (forward && dn.pq) {   // screen into the pair cache, then stream it
        const tmd_status st = launch_screen(dm, dn, s);
        if (st != TMD_OK) return st;
        if (dm.rtab)
            TMD_LAUNCH("k_desc", s, k_desc<K, S, true, true><<<nblk, PW * 32, 0, s>>>(dm, dn, pos, types, nl->G, nl->P));
        else
            TMD_LAUNCH("k_desc", s, k_desc<K, S, false, true><<<nblk, PW * 32, 0, s>>>(dm, dn, pos, types, nl->G, nl->P));
    } else if (forward && dm.rtab)
        TMD_LAUNCH("k_desc", s, k_desc<K, S, true, false><<<nblk, PW * 32, 0, s>>>(dm, dn, pos, types, nl->G, nl->P));
    else if (forward)
        TMD_LAUNCH("k_desc", s, k_desc<K, S, false, false><<<nblk, PW * 32, 0, s>>>(dm, dn, pos, types, nl->G, nl->P));
    else if (w_atom && dm.rtab)   // batched evaluations always run with the pair cache
        TMD_LAUNCH("k_force", s, k_force<K, S, true, true, true><<<nblk, PW * 32, 0, s>>>(dm, dn, pos, types, nl->P,
                                                                                        nl->dG, nl->Fq, part_w, w_atom));
    else if (w_atom)
        TMD_LAUNCH("k_force", s, k_force<K, S, true, true, false><<<nblk, PW * 32, 0, s>>>(dm, dn, pos, types, nl->P,
                                                                                         nl->dG, nl->Fq, part_w, w_atom));
    // the tensor-core pass reads the pair cache; an evaluation without one
    // (the allocation-free call) runs the SIMT pass whatever the setting
    else if (force_kernel() == TMD_FORCE_TENSOR && dn.pq && !(!dm.rtab && S == 1 && K <= 32)) {
        set_error("the tensor-core force pass needs one species, K <= 32 and the direct radial basis");
        return TMD_ERR_UNIMPLEMENTED;
    } else if (force_kernel() == TMD_FORCE_TENSOR && dn.pq) {
        if constexpr (S == 1 && K <= 32)
            TMD_LAUNCH("k_force", s, k_force_tc<K><<<nblk, PW * 32, 0, s>>>(dm, dn, nl->P, nl->dG, nl->Fq, part_w));
    } else if (dn.pq && dm.rtab)
        TMD_LAUNCH("k_force", s, k_force_merged<K, S, true><<<nblk, PW * 32, 0, s>>>(dm, dn, types, nl->P, nl->dG,
                                                                                   nl->Fq, part_w));
    else if (dn.pq)
        TMD_LAUNCH("k_force", s, k_force_merged<K, S, false><<<nblk, PW * 32, 0, s>>>(dm, dn, types, nl->P, nl->dG,
                                                                                    nl->Fq, part_w));
    else if (dm.rtab)
        TMD_LAUNCH("k_force", s, k_force<K, S, false, false, true><<<nblk, PW * 32, 0, s>>>(dm, dn, pos, types, nl->P,
                                                                                          nl->dG, nl->Fq, part_w, nullptr));
    else
        TMD_LAUNCH("k_force", s, k_force<K, S, false, false, false><<<nblk, PW * 32, 0, s>>>(dm, dn, pos, types, nl->P,
                                                                                           nl->dG, nl->Fq, part_w, nullptr));
    TMD_CUDA(cudaGetLastError());
    return TMD_OK;
}

}  // namespace

}  // namespace tmd
