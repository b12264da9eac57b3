// sdm_kernels.cuh -- CUDA kernels of one SDM coalescence timestep (sm_103a).
//
// A timestep (Fig. "fig:algo") runs each cell's Steps 0-3 inside one kernel
// kind chosen by the cell's width, so that only the data a decision needs is
// read and only changed super-droplets are written:
//
//  warp_cells_kernel  one warp per cell of at most 512 slots (the grid
//                     workloads): the cell's one-byte volume bins into shared
//                     memory, the shuffled list (Philox keys and a counting
//                     sort for up to 256 live SDs, else the keyed bijection
//                     from per-cell round tables), then per pair phi and the
//                     early exit against a bound of p; the pairs it cannot
//                     settle go to the step's queue.
//  wc_pairs_kernel    the queued pairs, one per thread: Steps 2-3 (certified
//                     FP32 interval, FP64 filters) and the update.
//  wc_compact_kernel  Step 0 of the cells the queued pairs emptied slots of.
//  tile_step_kernel   one CTA per run of cells between 512 slots and the
//                     schedule's tile size: the same steps with the tile's
//                     multiplicities and volumes in shared memory.
//  big_prp_kernel     cells above the tile size under the PRP contract: one
//                     cooperative wave over all of them, each thread mapping
//                     list positions through the keyed bijection, gathering the
//                     volume bins, settling most pairs by the early exit and
//                     queueing the rest per warp; Step 0 of cells flagged by the
//                     previous launch runs first, behind a bounded grid barrier.
//  big_scatter_kernel / big_finish_kernel
//                     the same cells under the SORT contract: the first pass
//                     scatters (key, position) records into fixed-capacity
//                     buckets by the key's top bits and writes each bucket's
//                     plan (its start in the cell's order); the second, one
//                     warp per bucket with the records staged by bulk copies,
//                     orders each bucket and takes its pairs through the early
//                     exit; the surviving pairs go to the step's queue (the
//                     allocation-free step's form evaluates them in the
//                     finishing warps).
//
// Every path realises the same shuffled list of the random-number contract
// (sort by (key, position), or the keyed bijection), so the tile size, bucket
// width and launch shape never change a result.
#pragma once
#include <utility>

#include "sdm_math.cuh"
#include "sdm_surrogate.cuh"

namespace sdm {

enum : uint32_t {
    ERR_BUCKET_OVERFLOW = 1u,
    ERR_TILE_OVERFLOW = 2u,
    ERR_TIMEOUT = 4u,
};

constexpr uint32_t PREC_FP64 = 0, PREC_FP32 = 1, PREC_SURROGATE = 2;
constexpr uint32_t SHUFFLE_PRP = 0, SHUFFLE_SORT = 1;
constexpr uint32_t DEAD = 0xffffffffu;

struct StepArgs {
    uint64_t* xi;
    double* attr;               // [n_attr][stride], attr 0 = volume
    uint8_t* vbin;              // [stride] vbin_of(volume) of every slot, kept current by every
                                // writer of the volumes; nullptr: not kept
    uint64_t stride;
    uint32_t n_attr;
    uint32_t precision;
    const uint32_t* cell_start; // [n_cell + 1]
    const double* dv;           // [n_cell]
    const uint8_t* kid;         // [n_cell]
    double dt;
    double golovin_b;
    double efield;              // field parameter of the electric-field kernel, in [0, 1]
    float dt_f;                 // dt, golovin_b and efield rounded to float on the host
    float golovin_bf;
    float efield_f;
    uint32_t seed_lo, seed_hi;
    PhiloxKeys pk;              // the key schedule of (seed_lo, seed_hi)
    uint32_t step;              // used when d_step == nullptr
    uint32_t shuffle;           // SHUFFLE_PRP or SHUFFLE_SORT
    const uint32_t* d_step;
    uint32_t* n_live;           // [n_cell] live SDs per cell (a prefix of its slots)
    const unsigned long long* cell_xmax;   // [n_cell] bound of the cell's multiplicities (small cells)
    unsigned long long* stats;  // [5] or nullptr
    uint32_t* err;
    const SurrogateDev* surr;   // device copy; used when precision == PREC_SURROGATE
    uint32_t stage_extra;       // failure-path self-test: bytes a staged bucket's copy announces
                                // beyond those it delivers (0: none; the wait then runs out)
    uint32_t wait_log2;         // bounded waits of the staged copies: 2^wait_log2 SM cycles (0: default)
};

// a cell is shuffled by sorting keys when it is small or the SORT contract is selected
__device__ __forceinline__ bool sorts(const StepArgs& a, uint32_t n)
{
    return a.shuffle == SHUFFLE_SORT || n < PRP_MIN_N;
}

struct TileDesc { uint32_t slot_begin, slot_end, cell_begin, n_cells; };
struct BigCell { uint32_t cell, slot_begin, width, bucket_base, nbits, quad_begin; };   // quad_begin: PRP contract
struct BigChunk { uint32_t big, l_begin, l_end, n_of_cell; };   // n_of_cell: chunks of the same cell
// per bucket of the SORT contract: what its finishing warp needs of its cell, in one 32-byte read
struct __align__(16) BucketDesc { uint32_t cell, slot_begin, bucket_base, nbits, big, pad0, pad1, pad2; };

__device__ __forceinline__ uint32_t step_index(const StepArgs& a)
{
    return a.d_step ? *a.d_step : a.step;
}

struct LocalStats {         // per thread; only the sum of gamma needs 64 bits
    uint32_t pairs, collisions, removed, fp64;
    unsigned long long sum_gamma;
};

struct CellCtx {
    uint32_t gid;      // global cell index
    uint32_t n;        // live SDs at the start of the step
    uint32_t kid;      // kernel id
    float s_dtdv32;    // pair-count ratio * dt / dV in FP32
    double dv;
};

// early-exit scale of a cell without its multiplicity factor (see pb_bin); with the
// surrogate the bound gets a factor 2 of room for the network's error
__device__ __forceinline__ float exit_scale(float s32, uint32_t kid, float golovin_bf, uint32_t precision)
{
    const float f = precision == PREC_SURROGATE ? 2.0f : 1.0f;
    return __fmul_ru(__fmul_ru(s32, kid == 0 ? golovin_bf : f), 1.0f + 0x1p-8f);
}

__device__ __forceinline__ float pair_ratio_dtdv_f(uint32_t n, float dt_f, double dv)
{
    // ((n^2 - n)/2) / floor(n/2) is n - 1 (n even) or n (n odd): exact integer
    const float s = (float)(n - 1u + (n & 1u));
    return s * (dt_f / d2f_trunc(dv));
}

// phi integers of candidate pairs 2M and 2M+1 of a cell (one Philox call)
__device__ __forceinline__ void phi_pair_u53(const StepArgs& a, uint32_t cell, uint32_t step, uint32_t M,
                                             uint64_t& u0, uint64_t& u1)
{
    const U4 x = philox(M, cell, step, 1u, a.pk);
    u0 = ((((uint64_t)x.x) << 32) | (uint64_t)x.y) >> 11;
    u1 = ((((uint64_t)x.z) << 32) | (uint64_t)x.w) >> 11;
}

// Step 2 + Step 3 for one candidate pair (first, second) of a cell with phi
// integer u53.  Writes the updated multiplicities and attributes of the pair to
// global memory.
// Kh_in: the surrogate's K^ of the pair when the caller evaluated it for the whole warp (-1: the
// plain kernel), or SURR_PER_LANE to evaluate it here
constexpr float SURR_PER_LANE = -2.0f;
template <bool SURR>
__device__ __forceinline__ void process_pair(const StepArgs& a, const EffTab* __restrict__ T, const CellCtx& c,
                                             uint64_t u53, uint64_t g1, uint64_t g2, uint64_t x1, uint64_t x2,
                                             double v1, double v2, LocalStats& ls, uint32_t* removed_flag,
                                             float Kh_in = SURR_PER_LANE)
{
    const bool swap = x1 < x2;                 // j = first unless it has the smaller multiplicity
    const uint64_t xj = swap ? x2 : x1, xk = swap ? x1 : x2;
    const float scale32 = u64_to_f_trunc(xj) * c.s_dtdv32;
    uint64_t g;
    float Kh = -1.0f;
    if (SURR && a.precision == PREC_SURROGATE && c.kid == 1)
        Kh = Kh_in != SURR_PER_LANE ? Kh_in : surr_pair_kernel(a.surr, v1, v2);
    const P32 pe = Kh >= 0.0f ? P32{Kh * scale32, 0.0f}
                              : pair_prob_f(T, c.kid, v1, v2, scale32, a.golovin_bf, a.efield_f);
    if (a.precision != PREC_FP64) {
        g = gamma_tilde_f(pe.p, u53, xj, xk);
    } else if (!gamma_tilde_certified(pe, u53, xj, xk, &g)) {
        // the second filter serves the gravitational kernel; the others go to the exact sequence
        if (c.kid != 1 || !gamma_tilde_lite(v1, v2, c.n, a.dt, c.dv, u53, xj, xk, &g))
            g = gamma_tilde_fp64_path(c.kid, v1, v2, a.golovin_b, a.efield, c.n, a.dt, c.dv, u53, xj, xk);
        ls.fp64++;
    }
    ls.pairs++;
    if (g == 0) return;
    const uint64_t gj = swap ? g2 : g1, gk = swap ? g1 : g2;
    const double vj = swap ? v2 : v1, vk = swap ? v1 : v2;
    const double gd = __ull2double_rn(g);
    const uint64_t new_n = xj - g * xk;
    if (new_n > 0) {                                          // case 1, eq. (coal_attr_0)
        a.xi[gj] = new_n;
        const double nv = __dadd_rn(__dmul_rn(gd, vj), vk);
        a.attr[gk] = nv;
        if (a.vbin) a.vbin[gk] = (uint8_t)vbin_of(nv);
        for (uint32_t i = 1; i < a.n_attr; ++i) {
            double* A = a.attr + (uint64_t)i * a.stride;
            A[gk] = __dadd_rn(__dmul_rn(gd, A[gj]), A[gk]);
        }
    } else {                                                  // case 2, eq. (coal)
        const uint64_t h = xk / 2;
        a.xi[gj] = h;
        a.xi[gk] = xk - h;
        const double nv = __dadd_rn(__dmul_rn(gd, vj), vk);
        a.attr[gj] = nv;
        a.attr[gk] = nv;
        if (a.vbin) {
            const uint8_t k = (uint8_t)vbin_of(nv);
            a.vbin[gj] = k;
            a.vbin[gk] = k;
        }
        for (uint32_t i = 1; i < a.n_attr; ++i) {
            double* A = a.attr + (uint64_t)i * a.stride;
            const double t = __dadd_rn(__dmul_rn(gd, A[gj]), A[gk]);
            A[gj] = t;
            A[gk] = t;
        }
        if (h == 0) {
            ls.removed++;
            *removed_flag = 1u;     // the cell needs compaction after the step
        }
    }
    ls.collisions++;
    ls.sum_gamma += g;
}

// ---------------------------------------------------------------------------
// block helpers
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void flush_stats(const StepArgs& a, LocalStats& ls, unsigned long long* red)
{
    if (!a.stats) return;
    unsigned long long v[5] = {ls.pairs, ls.collisions, ls.removed, ls.sum_gamma, ls.fp64};
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const unsigned long long s = warp_sum(v[k]);
        if (lane == 0 && s) atomicAdd(&red[k], s);
    }
    __syncthreads();
    if (threadIdx.x < 5 && red[threadIdx.x]) atomicAdd(&a.stats[threadIdx.x], red[threadIdx.x]);
}

// Exclusive scan of a[0..n) in place (block-wide); warp_tot[32] receives the total, and a[n]
// too when store_total.  'warp_tot' needs 33 entries of shared memory.
__device__ void block_exclusive_scan(uint32_t* a, uint32_t n, uint32_t* warp_tot, bool store_total = true)
{
    const uint32_t nt = blockDim.x, tid = threadIdx.x;
    const uint32_t per = (n + nt - 1) / nt;
    const uint32_t b0 = min(n, tid * per), b1 = min(n, b0 + per);
    uint32_t s = 0;
    for (uint32_t i = b0; i < b1; ++i) s += a[i];
    // inclusive warp scan of the thread sums
    const int lane = tid & 31, wid = tid >> 5;
    uint32_t inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const uint32_t nw = (nt + 31) >> 5;
        uint32_t w = lane < (int)nw ? warp_tot[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < (int)nw) warp_tot[lane] = wi - w;     // exclusive warp offsets
        if (lane == 31) warp_tot[32] = wi;               // block total
    }
    __syncthreads();
    uint32_t run = warp_tot[wid] + inc - s;
    for (uint32_t i = b0; i < b1; ++i) {
        const uint32_t t = a[i];
        a[i] = run;
        run += t;
    }
    if (tid == 0 && store_total) a[n] = warp_tot[32];
    __syncthreads();
}

// largest c in [0, n) with pre[c] <= x (pre non-decreasing)
__device__ __forceinline__ uint32_t find_segment(const uint32_t* pre, uint32_t n, uint32_t x)
{
    uint32_t lo = 0, hi = n;   // invariant: pre[lo] <= x, answer in [lo, hi)
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pre[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

__host__ __device__ __forceinline__ uint32_t ceil_log2(uint32_t w)
{
#ifdef __CUDA_ARCH__
    return w <= 1 ? 0u : 32u - __clz(w - 1u);
#else
    return w <= 1 ? 0u : 32u - (uint32_t)__builtin_clz(w - 1u);
#endif
}

// ---------------------------------------------------------------------------
// Tile kernel: whole small cells in shared memory.
// ---------------------------------------------------------------------------
constexpr uint32_t TQ_CAP = 96;   // tile kernel: queued pairs per warp (< 32 left + 2 x 32 new)
struct TileQueue {                 // local slots of the pair, cell index in the tile, phi integer
    uint32_t ii[TQ_CAP], c[TQ_CAP];
    unsigned long long u[TQ_CAP];
};

struct TileLayout {
    uint32_t tile_slots, max_cells;
    // byte offsets
    uint32_t o_xi, o_v, o_key, o_bo, o_cnt, o_tmp, o_srt, o_cs, o_gb, o_bb, o_pb, o_ss, o_nb, o_n, o_rem, o_pp, o_ctx, o_red,
        o_wt, o_tab, o_cup, o_q, o_prp;
    uint32_t bytes;
};

__host__ __device__ inline uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline TileLayout tile_layout(uint32_t tile_slots, uint32_t max_cells, uint32_t n_warps)
{
    TileLayout L;
    L.tile_slots = tile_slots;
    L.max_cells = max_cells;
    uint32_t o = 0;
    L.o_xi = o;  o = align_up(o + 8 * tile_slots, 16);
    L.o_v = o;   o = align_up(o + 8 * tile_slots, 16);
    L.o_key = o; o = align_up(o + 4 * tile_slots, 16);
    L.o_bo = o;  o = align_up(o + 4 * tile_slots, 16);
    L.o_cnt = o; o = align_up(o + 4 * (2 * tile_slots + 1), 16);
    L.o_tmp = o; o = align_up(o + 2 * tile_slots, 16);
    L.o_srt = o; o = align_up(o + 2 * tile_slots, 16);
    L.o_cs = o;  o = align_up(o + 4 * (max_cells + 1), 16);
    L.o_gb = o;  o = align_up(o + 4 * (max_cells + 1), 16);
    L.o_bb = o;  o = align_up(o + 4 * (max_cells + 1), 16);
    L.o_pb = o;  o = align_up(o + 4 * (max_cells + 1), 16);
    L.o_ss = o;  o = align_up(o + 4 * (max_cells + 1), 16);
    L.o_nb = o;  o = align_up(o + 4 * (max_cells + 1), 16);
    L.o_n = o;   o = align_up(o + 4 * (max_cells + 1), 16);
    L.o_rem = o; o = align_up(o + 4 * (max_cells + 1), 16);
    L.o_pp = o;  o = align_up(o + 4 * (max_cells + 1), 16);
    L.o_ctx = o; o = align_up(o + (uint32_t)sizeof(CellCtx) * max_cells, 16);
    L.o_red = o; o = align_up(o + 8 * 8, 16);
    L.o_wt = o;  o = align_up(o + 4 * 40, 16);
    L.o_tab = o; o = align_up(o + (uint32_t)sizeof(EffTab), 16);
    L.o_cup = o; o = align_up(o + 4 * (max_cells + 1), 16);
    // the bijections of the tile's cells above PRP_MIN_N SDs (at most tile_slots / PRP_MIN_N)
    L.o_prp = o; o = align_up(o + (uint32_t)sizeof(Prp) * (tile_slots / PRP_MIN_N + 1), 16);
    // the pair queues live in the sort scratch (keys, bucket offsets, counts, tmp), which is
    // dead once the shuffled lists are built
    const uint32_t qbytes = (uint32_t)sizeof(TileQueue) * n_warps;
    if (qbytes <= L.o_srt - L.o_key) {
        L.o_q = L.o_key;
    } else {
        L.o_q = o;   o = align_up(o + qbytes, 16);
    }
    L.bytes = o;
    return L;
}

// warp 0 computes an exclusive scan over n (<= max_cells) values in place; a[n] = total
__device__ __forceinline__ void warp0_exclusive_scan(uint32_t* a, uint32_t n)
{
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    uint32_t carry = 0;
    for (uint32_t base = 0; base < n; base += 32) {
        const uint32_t i = base + lane;
        const uint32_t v = i < n ? a[i] : 0u;
        uint32_t inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (i < n) a[i] = carry + inc - v;
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) a[n] = carry;
}

// the same for three arrays at once (independent shuffle chains, one pass)
__device__ __forceinline__ void warp0_exclusive_scan3(uint32_t* a, uint32_t* b, uint32_t* c, uint32_t n)
{
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    uint32_t ca = 0, cb = 0, cc = 0;
    for (uint32_t base = 0; base < n; base += 32) {
        const uint32_t i = base + lane;
        const uint32_t va = i < n ? a[i] : 0u, vb = i < n ? b[i] : 0u, vc = i < n ? c[i] : 0u;
        uint32_t ia = va, ib = vb, ic = vc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t ta = __shfl_up_sync(0xffffffffu, ia, o);
            const uint32_t tb = __shfl_up_sync(0xffffffffu, ib, o);
            const uint32_t tc = __shfl_up_sync(0xffffffffu, ic, o);
            if (lane >= o) { ia += ta; ib += tb; ic += tc; }
        }
        if (i < n) { a[i] = ca + ia - va; b[i] = cb + ib - vb; c[i] = cc + ic - vc; }
        ca += __shfl_sync(0xffffffffu, ia, 31);
        cb += __shfl_sync(0xffffffffu, ib, 31);
        cc += __shfl_sync(0xffffffffu, ic, 31);
    }
    if (lane == 0) { a[n] = ca; b[n] = cb; c[n] = cc; }
}

// Stable compaction of one cell by one warp: the live SDs of slots
// [base, base + n_old) move, in order, to the front; the freed slots get xi = 0
// and attributes 0.  Attribute rows move first (liveness is read from xi, which
// moves last); within a chunk of 32 every lane reads before any lane writes, and
// a destination never lies after its source.  Returns the new live count.
__device__ uint32_t warp_compact_cell(const StepArgs& a, uint64_t base, uint32_t n_old, uint32_t lane)
{
    const unsigned lt = (1u << lane) - 1u;
    uint32_t dst = 0;
    for (uint32_t r = 0; r <= a.n_attr; ++r) {
        dst = 0;
        for (uint32_t off = 0; off < n_old; off += 32) {
            const uint32_t i = off + lane;
            const bool in = i < n_old;
            const uint64_t x = in ? a.xi[base + i] : 0ull;
            const bool live = x != 0;
            const unsigned mask = __ballot_sync(0xffffffffu, live);
            const uint32_t pos = dst + __popc(mask & lt);
            if (r < a.n_attr) {
                double* A = a.attr + (uint64_t)r * a.stride + base;
                const double v = in ? A[i] : 0.0;
                __syncwarp();
                if (live) {
                    A[pos] = v;
                    if (r == 0 && a.vbin) a.vbin[base + pos] = (uint8_t)vbin_of(v);
                }
            } else {
                __syncwarp();
                if (live) a.xi[base + pos] = x;
            }
            dst += __popc(mask);
            __syncwarp();
        }
    }
    for (uint32_t i = dst + lane; i < n_old; i += 32) {
        a.xi[base + i] = 0ull;
        for (uint32_t r = 0; r < a.n_attr; ++r) a.attr[(uint64_t)r * a.stride + base + i] = 0.0;
        if (a.vbin) a.vbin[base + i] = 0;
    }
    __syncwarp();
    return dst;
}

template <bool SURR>
__device__ void tile_process(const StepArgs& a, const TileDesc td, const TileLayout& L, unsigned char* smem,
                             uint32_t step, LocalStats& ls)
{
    uint64_t* xi_s = (uint64_t*)(smem + L.o_xi);
    double* v_s = (double*)(smem + L.o_v);
    uint32_t* key_s = (uint32_t*)(smem + L.o_key);
    uint32_t* bo_s = (uint32_t*)(smem + L.o_bo);
    uint32_t* cnt = (uint32_t*)(smem + L.o_cnt);
    uint16_t* tmp = (uint16_t*)(smem + L.o_tmp);
    uint16_t* srt = (uint16_t*)(smem + L.o_srt);
    uint32_t* cs = (uint32_t*)(smem + L.o_cs);
    uint32_t* gb = (uint32_t*)(smem + L.o_gb);
    uint32_t* bb = (uint32_t*)(smem + L.o_bb);
    uint32_t* pb = (uint32_t*)(smem + L.o_pb);
    uint32_t* ss = (uint32_t*)(smem + L.o_ss);
    uint32_t* nbit = (uint32_t*)(smem + L.o_nb);
    uint32_t* ncl = (uint32_t*)(smem + L.o_n);
    uint32_t* rem = (uint32_t*)(smem + L.o_rem);
    uint32_t* pp = (uint32_t*)(smem + L.o_pp);
    CellCtx* ctx = (CellCtx*)(smem + L.o_ctx);
    uint32_t* wt = (uint32_t*)(smem + L.o_wt);
    const EffTab* tab = (const EffTab*)(smem + L.o_tab);
    float* cup = (float*)(smem + L.o_cup);

    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    const uint32_t ns = td.slot_end - td.slot_begin, nc = td.n_cells;

    // per cell: slot offset, live count (the live SDs are the first n slots), and
    // what Step 1 needs: key groups and buckets for sorted cells, the list length
    // for PRP-shuffled cells
    if (tid == 0) {
        wt[39] = 0;                 // PRP cells of the tile, counted when their bijections are set up
        wt[38] = 0;                 // their positions whose first image walks
    }
    for (uint32_t c = tid; c <= nc; c += nt) {
        cs[c] = a.cell_start[td.cell_begin + c] - td.slot_begin;
        if (c < nc) {
            const uint32_t w = a.cell_start[td.cell_begin + c + 1] - a.cell_start[td.cell_begin + c];
            const uint32_t n = min(a.n_live[td.cell_begin + c], w);
            const bool srt_c = sorts(a, n);
            ncl[c] = n;
            rem[c] = 0;
            const uint32_t nb = ceil_log2(n);
            nbit[c] = nb;
            gb[c] = srt_c ? (n + 3) >> 2 : 0u;
            bb[c] = (srt_c && n) ? 1u << nb : 0u;      // 2^ceil(log2 n) <= 2n buckets
            pp[c] = srt_c ? 0u : n;
            ctx[c].kid = a.kid[td.cell_begin + c];      // loaded with the slots, used after the sort
            ctx[c].dv = a.dv[td.cell_begin + c];
        }
    }
    // the tile's multiplicities and volumes: every load of a thread in flight before its stores
    constexpr uint32_t LB = 4;
    for (uint32_t i0 = tid; i0 < ns; i0 += LB * nt) {
        uint64_t xr[LB];
        double vr[LB];
#pragma unroll
        for (uint32_t k = 0; k < LB; ++k) {
            const uint32_t i = i0 + k * nt;
            if (i < ns) {
                xr[k] = a.xi[td.slot_begin + i];
                vr[k] = a.attr[td.slot_begin + i];
            }
        }
#pragma unroll
        for (uint32_t k = 0; k < LB; ++k) {
            const uint32_t i = i0 + k * nt;
            if (i < ns) {
                xi_s[i] = xr[k];
                v_s[i] = vr[k];
            }
        }
    }
    __syncthreads();
    if (tid < 32) warp0_exclusive_scan3(gb, bb, pp, nc);
    __syncthreads();
    const uint32_t G = gb[nc], NB = bb[nc];
    for (uint32_t b = tid; b < NB; b += nt) cnt[b] = 0;
    for (uint32_t i = tid; i < ns; i += nt) bo_s[i] = DEAD;
    __syncthreads();

    // Step 1 for sorted cells: Philox keys of the list positions, bucket counts
    for (uint32_t g = tid; g < G; g += nt) {
        const uint32_t c = find_segment(gb, nc, g);
        const uint32_t grp = g - gb[c];
        const uint32_t n = ncl[c];
        const U4 x = philox(grp, td.cell_begin + c, step, 0u, a.pk);
        const uint32_t nb = nbit[c];
#pragma unroll
        for (uint32_t k = 0; k < 4; ++k) {
            const uint32_t l = 4 * grp + k;
            if (l >= n) break;
            const uint32_t i = cs[c] + l;
            const uint32_t key = u4_word(x, k);
            const uint32_t b = bb[c] + (nb ? key >> (32u - nb) : 0u);
            const uint32_t off = atomicAdd(&cnt[b], 1u);
            key_s[i] = key;
            bo_s[i] = (b << 16) | off;
        }
    }
    __syncthreads();
    block_exclusive_scan(cnt, NB, wt);
    for (uint32_t i = tid; i < ns; i += nt) {
        const uint32_t bo = bo_s[i];
        if (bo != DEAD) tmp[cnt[bo >> 16] + (bo & 0xffffu)] = (uint16_t)i;
    }
    __syncthreads();
    // exact rank inside the bucket: order by (key, list position)
    for (uint32_t i = tid; i < ns; i += nt) {
        const uint32_t bo = bo_s[i];
        if (bo == DEAD) continue;
        const uint32_t b = bo >> 16;
        const uint32_t st = cnt[b], en = cnt[b + 1];
        const uint32_t key = key_s[i];
        uint32_t r = 0;
        for (uint32_t p = st; p < en; ++p) {
            const uint32_t o = tmp[p];
            const uint32_t ko = key_s[o];
            r += (ko < key) || (ko == key && o < i);
        }
        srt[st + r] = (uint16_t)i;
    }
    // where each cell's shuffled list starts in srt; per-cell constants of eq. (p)
    Prp* prp_s = (Prp*)(smem + L.o_prp);
    for (uint32_t c = tid; c < nc; c += nt) {
        const uint32_t n = ncl[c];
        ss[c] = sorts(a, n) ? cnt[bb[c]] : NB ? cnt[NB] + pp[c] : pp[c];
        if (!sorts(a, n)) {
            // the cell's bijection, once: its index among the tile's PRP cells replaces the
            // bucket bit count, which only sorted cells use
            const uint32_t k = atomicAdd(&wt[39], 1u);
            prp_init(prp_s[k], a.pk, td.cell_begin + c, step, n);
            nbit[c] = k;
        }
        const uint32_t gid = td.cell_begin + c;
        CellCtx cc = ctx[c];                         // kid and dv, loaded with the slots
        cc.gid = gid;
        cc.n = n;
        cc.s_dtdv32 = n >= 2 ? pair_ratio_dtdv_f(n, a.dt_f, cc.dv) : 0.f;
        ctx[c] = cc;
        cup[c] = exit_scale(cc.s_dtdv32, cc.kid, a.golovin_bf, a.precision);
        pb[c] = (n >> 1) + 1u >> 1;              // groups of two pairs (one Philox call each)
    }
    __syncthreads();
    // Step 1 for the larger cells under the PRP contract: L'[q] = L[P(q)], every position of
    // every such cell of the tile in one pass
    // every position of every such cell of the tile in one pass.  A first image outside [0, n)
    // goes to a list (position | image << 13; the bucket offsets' memory is free by now) that
    // full warps walk afterwards, instead of holding its warp for a second pass of the network
    const uint32_t NPE = pp[nc];
    uint32_t* walk = bo_s;
    for (uint32_t t = tid; t < NPE; t += nt) {
        const uint32_t c = find_segment(pp, nc, t);
        const uint32_t q = t - pp[c];
        const Prp& P = prp_s[nbit[c]];
        const uint32_t e = feistel(P, q);
        if (e < P.n) srt[ss[c] + q] = (uint16_t)(cs[c] + e);
        else walk[atomicAdd(&wt[38], 1u)] = t | (e << 13);
    }
    __syncthreads();
    const uint32_t NW = wt[38];
    for (uint32_t k = tid; k < NW; k += nt) {
        const uint32_t t = walk[k] & 0x1fffu;
        uint32_t e = walk[k] >> 13;
        const uint32_t c = find_segment(pp, nc, t);
        const Prp& P = prp_s[nbit[c]];
        do e = feistel(P, e); while (e >= P.n);
        srt[ss[c] + t - pp[c]] = (uint16_t)(cs[c] + e);
    }
    if (tid < 32) warp0_exclusive_scan(pb, nc);
    __syncthreads();
    const uint32_t P2 = pb[nc];
    // Steps 2-3 for every candidate pair of the tile, two consecutive pairs per thread.  Most
    // pairs are settled by the early exit (phi above a bound of p); the others are queued per
    // warp and evaluated 32 at a time.
    const uint32_t lane = tid & 31;
    TileQueue& Q = ((TileQueue*)(smem + L.o_q))[tid >> 5];
    uint32_t qcnt = 0;                                         // warp-uniform
    for (uint32_t base = tid & ~31u; base < P2; base += nt) {  // warp-uniform trip count
        const uint32_t t = base + lane;
        const bool valid = t < P2;
        const uint32_t c = valid ? find_segment(pb, nc, t) : 0u;
        const uint32_t M = valid ? t - pb[c] : 0u;
        const CellCtx& cc = ctx[c];
        U4 w = {0, 0, 0, 0};
        if (valid) w = philox(M, cc.gid, step, 1u, a.pk);
        const float* __restrict__ tb = g_pbound[cc.kid];
#pragma unroll
        for (uint32_t h = 0; h < 2; ++h) {
            const uint32_t m = 2 * M + h;
            const bool has = valid && m < (cc.n >> 1);
            bool need = false;
            uint32_t i1 = 0, i2 = 0;
            const uint32_t whi = h ? w.z : w.x, wlo = h ? w.w : w.y;
            if (has) {
                i1 = srt[ss[c] + 2 * m];
                i2 = srt[ss[c] + 2 * m + 1];
                const float pup = __fmul_ru(__fmul_ru(__ldg(tb + pb_index(vbin_of(v_s[i1]), vbin_of(v_s[i2]))),
                                                      cup[c]),
                                            xi_pow2_above(xi_s[i1], xi_s[i2]));
                need = !(pup <= phi_lo23(whi));
                ls.pairs += need ? 0u : 1u;
            }
            const unsigned mk = __ballot_sync(0xffffffffu, need);
            if (need) {
                const uint32_t k = qcnt + __popc(mk & ((1u << lane) - 1u));
                Q.ii[k] = i1 | (i2 << 16);
                Q.c[k] = c;
                Q.u[k] = ((((uint64_t)whi) << 32) | (uint64_t)wlo) >> 11;
            }
            qcnt += __popc(mk);
        }
        while (qcnt >= 32) {
            __syncwarp();
            const uint32_t k = qcnt - 32 + lane;
            const uint32_t ii = Q.ii[k], cq = Q.c[k];
            const uint32_t i1 = ii & 0xffffu, i2 = ii >> 16;
            float Kh = SURR_PER_LANE;
            if (SURR && a.precision == PREC_SURROGATE)        // the warp's pairs on the tensor cores
                Kh = surr_pair_kernel_warp(a.surr, v_s[i1], v_s[i2], ctx[cq].kid == 1);
            process_pair<SURR>(a, tab, ctx[cq], Q.u[k], td.slot_begin + i1, td.slot_begin + i2, xi_s[i1], xi_s[i2],
                         v_s[i1], v_s[i2], ls, &rem[cq], Kh);
            __syncwarp();
            qcnt -= 32;
        }
    }
    __syncwarp();
    {
        const bool act = lane < qcnt;
        const uint32_t ii = act ? Q.ii[lane] : 0u, cq = act ? Q.c[lane] : 0u;
        const uint32_t i1 = ii & 0xffffu, i2 = ii >> 16;
        float Kh = SURR_PER_LANE;
        if (SURR && a.precision == PREC_SURROGATE)
            Kh = surr_pair_kernel_warp(a.surr, v_s[i1], v_s[i2], act && ctx[cq].kid == 1);
        if (act)
            process_pair<SURR>(a, tab, ctx[cq], Q.u[lane], td.slot_begin + i1, td.slot_begin + i2, xi_s[i1],
                               xi_s[i2], v_s[i1], v_s[i2], ls, &rem[cq], Kh);
    }
    __syncthreads();
    // removals take effect in storage: compact the cells that lost SDs (rare)
    const uint32_t warp = tid >> 5, nw = nt >> 5;
    for (uint32_t c = warp; c < nc; c += nw) {
        if (!rem[c]) continue;
        const uint32_t n_new = warp_compact_cell(a, td.slot_begin + cs[c], ncl[c], lane);
        if (lane == 0) a.n_live[td.cell_begin + c] = n_new;
    }
}

#ifndef SDM_TILE_MIN_BLOCKS
#define SDM_TILE_MIN_BLOCKS 4
#endif
// MAXT: the largest block the instantiation takes (256: SDM_TILE_MIN_BLOCKS resident blocks of
// 256 threads per SM, registers permitting; 512: one block)
template <bool SURR, uint32_t MAXT>
__global__ void __launch_bounds__(MAXT, MAXT <= 256 ? SDM_TILE_MIN_BLOCKS : 1) tile_step_kernel(StepArgs a, const TileDesc* __restrict__ tiles,
                                                         uint32_t n_tiles, TileLayout L, uint32_t* work)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t step = step_index(a);
    LocalStats ls = {0, 0, 0, 0, 0ull};
    unsigned long long* red = (unsigned long long*)(smem + L.o_red);
    load_eff_tab((EffTab*)(smem + L.o_tab));   // read after the first __syncthreads of tile_process
    if (work == nullptr) {
        tile_process<SURR>(a, tiles[blockIdx.x], L, smem, step, ls);
    } else {
        __shared__ uint32_t t_s;
        for (;;) {
            if (threadIdx.x == 0) t_s = atomicAdd(&work[0], 1u);
            __syncthreads();
            const uint32_t t = t_s;
            __syncthreads();
            if (t >= n_tiles) break;
            tile_process<SURR>(a, tiles[t], L, smem, step, ls);
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            __threadfence();
            const uint32_t done = atomicAdd(&work[1], 1u);
            if (done == gridDim.x - 1) { work[0] = 0; work[1] = 0; __threadfence(); }
        }
    }
    if (a.stats) {
        __syncthreads();
        if (threadIdx.x < 5) red[threadIdx.x] = 0;
        __syncthreads();
        flush_stats(a, ls, red);
    }
}

// ---------------------------------------------------------------------------
// Small cells, one warp per cell.  A cell of at most WC_MAX slots is stepped by
// one warp with no block barrier: the warp reads the volume bins of the cell's
// SDs (one byte each) into shared memory, builds the shuffled list (a counting
// sort of the Philox keys by their top bits, the keys sharing a bucket ordered
// within it, or the keyed bijection for a cell above 256 SDs under the PRP
// contract), settles pairs by the early exit against the cell's multiplicity
// bound and appends the others to the step's queue, which wc_pairs_kernel
// evaluates (wc_compact_kernel then compacts the cells that lost an SD).  Many
// independent warps per SM hide each other's latencies.
// ---------------------------------------------------------------------------
constexpr uint32_t WC_MAX = 512;          // slots of a cell stepped by one warp
constexpr uint32_t WC_WARPS = 4;          // warps per block
constexpr uint32_t WC_TAB = 32;           // entries per round table of the bijection (A, B <= 32 for n <= 512)
constexpr uint32_t WC_SORT_PRP = PRP_MIN_N - 1;   // longest list sorted by key under the PRP contract
#ifndef SDM_WC_MIN_BLOCKS
#define SDM_WC_MIN_BLOCKS 9
#endif

// Per-warp shared memory of the small-cell step.  SMAX: the longest list the warp sorts by key
// (PRP_MIN_N - 1 under the PRP contract, whose longer lists take the bijection; WC_MAX under the
// SORT contract).
template <uint32_t SMAX>
struct __align__(16) WarpCellSmem {
    union __align__(16) {
        struct {                          // Step 1 by sorting keys (n <= SMAX)
            uint32_t key[SMAX];
            uint16_t cnt[(SMAX <= 256 ? 2 : 1) * SMAX + 2];   // bucket counts (warp_sort_keys), then offsets
            uint16_t off[SMAX];           // a position's place in its bucket's arrival order
            uint16_t tmp[SMAX];           // positions grouped by bucket
        } s;
        struct {                          // Step 1 by the keyed bijection (257 <= n <= WC_MAX)
            uint8_t tab[PRP_ROUNDS][WC_TAB];   // round r: floor(h(v ^ Kx_r) M_r / 2^32) for v < 32
            uint32_t walk[WC_TAB];        // positions whose image lies outside [0, n) (fewer than A)
        } p;
    };
    uint16_t srt[WC_MAX];                 // the shuffled list: offsets in the cell
    uint8_t vb[WC_MAX];                   // bin of each SD's volume (the state's vbin)
};

// The queue of the small-cell step: pairs that passed the early exit, 16 bytes each (cell,
// offsets i1 | i2 << 16 of the two SDs in the cell, and the pair's phi integer), appended by
// warp_cells_kernel and evaluated by wc_pairs_kernel; cells that lost an SD are listed for
// wc_compact_kernel.  The counters are zero between steps (the compaction kernel resets them).
constexpr uint32_t WQ_BIG = 0x80000000u;    // pair index flag: a large cell's pair
struct WcQueue {
    uint4* q;                 // [capacity] (cell, slot of the first SD, slot of the second, pair index m
                              // of the cell | WQ_BIG for a large cell); phi_m is recomputed from m
    uint32_t* count;          // [0] queued pairs, [1] listed cells of one warp, [2] the compaction
                              // kernel's ticket, [3] listed large cells
    uint32_t* cells;          // [cells of one warp] cells to compact
    uint32_t* bigcells;       // [large cells] large cells to compact
    uint32_t* flag;           // [n_cell] the cell is listed
};
__device__ uint32_t block_compact_cell(const StepArgs& a, uint64_t base, uint32_t n_old, uint32_t* wt);


// exclusive scan of a[0..n) by one warp; a[n] = total
__device__ __forceinline__ void warp_exclusive_scan(uint32_t* a, uint32_t n, uint32_t lane)
{
    const uint32_t per = (n + 31) >> 5;
    const uint32_t b0 = min(n, lane * per), b1 = min(n, b0 + per);
    uint32_t s = 0;
    for (uint32_t i = b0; i < b1; ++i) s += a[i];
    uint32_t inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= (uint32_t)o) inc += t;
    }
    uint32_t run = inc - s;
    for (uint32_t i = b0; i < b1; ++i) {
        const uint32_t t = a[i];
        a[i] = run;
        run += t;
    }
    const uint32_t tot = __shfl_sync(0xffffffffu, inc, 31);
    if (lane == 0) a[n] = tot;
    __syncwarp();
}

// The same on 16-bit entries whose total is below 2^15, for n = 32 * 2 W (W 32-bit words of two
// entries per lane, 16-byte aligned for W >= 4): one vector load and store per lane, the two halves
// of each word summed together (no carry between them, the total being below 2^15).
template <uint32_t W>
__device__ __forceinline__ void warp_exclusive_scan16_words(uint16_t* a, uint32_t n, uint32_t lane)
{
    uint32_t* base = reinterpret_cast<uint32_t*>(a) + lane * W;
    uint32_t w[W];
    if constexpr (W >= 4) {
#pragma unroll
        for (uint32_t c = 0; c < W / 4; ++c) {
            const uint4 v = reinterpret_cast<const uint4*>(base)[c];
            w[4 * c] = v.x; w[4 * c + 1] = v.y; w[4 * c + 2] = v.z; w[4 * c + 3] = v.w;
        }
    } else if constexpr (W == 2) {
        const uint2 v = *reinterpret_cast<const uint2*>(base);
        w[0] = v.x; w[1] = v.y;
    } else {
        w[0] = base[0];
    }
    uint32_t t = 0;
#pragma unroll
    for (uint32_t i = 0; i < W; ++i) t += w[i];
    const uint32_t s = (t & 0xffffu) + (t >> 16);
    uint32_t inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= (uint32_t)o) inc += u;
    }
    uint32_t run = inc - s;
#pragma unroll
    for (uint32_t i = 0; i < W; ++i) {
        const uint32_t lo = w[i] & 0xffffu, hi = w[i] >> 16;
        w[i] = run | ((run + lo) << 16);
        run += lo + hi;
    }
    if constexpr (W >= 4) {
#pragma unroll
        for (uint32_t c = 0; c < W / 4; ++c)
            reinterpret_cast<uint4*>(base)[c] = make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
    } else if constexpr (W == 2) {
        *reinterpret_cast<uint2*>(base) = make_uint2(w[0], w[1]);
    } else {
        base[0] = w[0];
    }
    if (lane == 31) a[n] = (uint16_t)run;
    __syncwarp();
}

// The same on 16-bit entries (totals below 2^15; a 16-byte aligned array when n >= 256): powers
// of two from 64 to 1024 take the vector form above.
__device__ __forceinline__ void warp_exclusive_scan16(uint16_t* a, uint32_t n, uint32_t lane)
{
    switch (n) {
    case 64: warp_exclusive_scan16_words<1>(a, n, lane); return;
    case 128: warp_exclusive_scan16_words<2>(a, n, lane); return;
    case 256: warp_exclusive_scan16_words<4>(a, n, lane); return;
    case 512: warp_exclusive_scan16_words<8>(a, n, lane); return;
    case 1024: warp_exclusive_scan16_words<16>(a, n, lane); return;
    default: break;
    }
    const uint32_t per = (n + 31) >> 5;
    const uint32_t b0 = min(n, lane * per), b1 = min(n, b0 + per);
    uint32_t s = 0;
    for (uint32_t i = b0; i < b1; ++i) s += a[i];
    uint32_t inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= (uint32_t)o) inc += t;
    }
    uint32_t run = inc - s;
    for (uint32_t i = b0; i < b1; ++i) {
        const uint32_t t = a[i];
        a[i] = (uint16_t)run;
        run += t;
    }
    const uint32_t tot = __shfl_sync(0xffffffffu, inc, 31);
    if (lane == 0) a[n] = (uint16_t)tot;
    __syncwarp();
}

// Step 1 by sorting keys: the list ordered by (key, position), key(l) = philox(l >> 2, c, s, 0)[l & 3].
// Counting sort on the top ceil(log2 n) + 1 bits for SMAX <= 256 (about one key per two buckets), else
// on the top ceil(log2 n) bits (about one per bucket; fewer registers): a key alone in its bucket
// goes straight to its place; the keys of a bucket holding several are grouped, the bucket is
// listed once, and each listed bucket is ordered by (key, position) with an insertion sort by one
// lane.  SMAX: the longest list (n <= SMAX), so that the per-key loops have fixed trip counts.
template <uint32_t SMAX, typename SM>
__device__ __forceinline__ void warp_sort_keys(const StepArgs& a, SM& S, uint32_t cell, uint32_t step, uint32_t n,
                                               uint32_t lane)
{
    constexpr uint32_t NI = (SMAX + 31) / 32;                  // keys per lane at most
    constexpr uint32_t NG = (SMAX + 127) / 128;                // Philox groups of four keys per lane at most
    const uint32_t nbb = ceil_log2(n) + (SMAX <= 256 ? 1u : 0u);   // n >= 2: 2^nbb >= n buckets
    const uint32_t sh = 32u - nbb;
    const uint32_t NBK = 1u << nbb;
    uint32_t* cw = reinterpret_cast<uint32_t*>(S.s.cnt);      // two 16-bit counts per word (n <= 512)
    for (uint32_t b = lane; 2 * b < NBK; b += 32) cw[b] = 0;
    __syncwarp();
#pragma unroll
    for (uint32_t j = 0; j < NG; ++j) {
        const uint32_t g = lane + 32 * j;
        if (4 * g < n) {
            const U4 x = philox(g, cell, step, 0u, a.pk);
            if (4 * g + 3 < n) *reinterpret_cast<uint4*>(&S.s.key[4 * g]) = make_uint4(x.x, x.y, x.z, x.w);
#pragma unroll
            for (uint32_t k = 0; k < 4; ++k) {
                const uint32_t l = 4 * g + k;
                if (l < n) {
                    const uint32_t key = u4_word(x, k);
                    if (4 * g + 3 >= n) S.s.key[l] = key;
                    const uint32_t b = key >> sh, hs = (b & 1u) << 4;   // count b: half b & 1 of word b >> 1
                    S.s.off[l] = (uint16_t)(atomicAdd(&cw[b >> 1], 1u << hs) >> hs);
                }
            }
        }
    }
    __syncwarp();
    warp_exclusive_scan16(S.s.cnt, NBK, lane);
    // singletons to their place; the others grouped by bucket in tmp, each such bucket listed once
    // (by its first arrival) in off: a list entry never lands on an arrival index still to be read
    uint32_t nwork = 0;
#pragma unroll
    for (uint32_t j = 0; j < NI; ++j) {
        if (32 * j >= n) break;                                 // uniform: the rest of the list is empty
        const uint32_t l = lane + 32 * j;
        bool lead = false;
        uint32_t b = 0;
        if (l < n) {
            b = S.s.key[l] >> sh;
            const uint32_t st = S.s.cnt[b], c = S.s.cnt[b + 1] - st;
            const uint32_t o = S.s.off[l];
            if (c == 1) S.srt[st] = (uint16_t)l;
            else S.s.tmp[st + o] = (uint16_t)l;
            lead = c > 1 && o == 0;
        }
        const unsigned m = __ballot_sync(0xffffffffu, lead);
        if (lead) S.s.off[nwork + __popc(m & ((1u << lane) - 1u))] = (uint16_t)b;
        nwork += __popc(m);
    }
    __syncwarp();
    for (uint32_t w = lane; w < nwork; w += 32) {
        const uint32_t b = S.s.off[w];
        const uint32_t st = S.s.cnt[b], en = S.s.cnt[b + 1];
        for (uint32_t i = st; i < en; ++i) {
            const uint32_t p = S.s.tmp[i], kp = S.s.key[p];
            uint32_t j = i;
            for (; j > st; --j) {
                const uint32_t q = S.srt[j - 1], kq = S.s.key[q];
                if (kq < kp || (kq == kp && q < p)) break;
                S.srt[j] = (uint16_t)q;
            }
            S.srt[j] = (uint16_t)p;
        }
    }
}

// The domain of the bijection (prp_domain_of) and ceil(2^32 / B) for every list length the
// small-cell step maps by it (PRP_MIN_N <= n <= WC_MAX), worked out at compile time: one
// constant-cache read per cell instead of a square root and two divisions.
struct PrpDom { uint32_t ab, binv; };      // ab = A | B << 16
constexpr PrpDom prp_dom_entry(uint32_t n)
{
    uint32_t A = 1, B = n;
    if ((n & (n - 1)) == 0) {
        uint32_t k = 0;
        while ((1u << k) < n) ++k;
        A = 1u << (k >> 1);
        B = 1u << (k - (k >> 1));
    } else {
        while (A * A < n) ++A;                 // ceil(sqrt n)
        B = (n + A - 1) / A;
    }
    return PrpDom{A | (B << 16), (uint32_t)((0x100000000ull + B - 1) / B)};
}
constexpr uint32_t PRP_DOM_N = WC_MAX - PRP_MIN_N + 1;
struct PrpDomTab { PrpDom e[PRP_DOM_N]; };
template <size_t... I>
constexpr PrpDomTab make_prp_dom_tab(std::index_sequence<I...>)
{
    return PrpDomTab{{prp_dom_entry(PRP_MIN_N + (uint32_t)I)...}};
}
__constant__ PrpDomTab c_prp_dom = make_prp_dom_tab(std::make_index_sequence<PRP_DOM_N>{});

// x mod M for x < 2 M, without a branch: x - M wraps around (becomes larger) when x < M
__device__ __forceinline__ uint32_t sub_mod(uint32_t x, uint32_t M) { return min(x, x - M); }

// The bijection's images of positions base + lane + 32 t, t < NT (the rounds of warp_prp_list;
// an image outside [0, n) goes to the walk list)
template <uint32_t NT, typename SM>
__device__ __forceinline__ void prp_positions(SM& S, uint32_t base, uint32_t n, uint32_t A, uint32_t B,
                                              uint32_t Binv, uint32_t& nwalk, uint32_t lane)
{
    uint32_t L[NT], R[NT];
#pragma unroll
    for (uint32_t t = 0; t < NT; ++t) {
        const uint32_t q = min(base + 32 * t + lane, n - 1);
        uint32_t h = __umulhi(q, Binv);
        if (h * B > q) --h;
        L[t] = h;
        R[t] = q - h * B;
    }
#pragma unroll
    for (uint32_t r = 0; r < PRP_ROUNDS; r += 2) {
#pragma unroll
        for (uint32_t t = 0; t < NT; ++t) L[t] = sub_mod(L[t] + S.p.tab[r][R[t]], A);
#pragma unroll
        for (uint32_t t = 0; t < NT; ++t) R[t] = sub_mod(R[t] + S.p.tab[r + 1][L[t]], B);
    }
#pragma unroll
    for (uint32_t t = 0; t < NT; ++t) {
        const uint32_t q = base + 32 * t + lane;
        const uint32_t e = L[t] * B + R[t];
        const bool walks = q < n && e >= n;
        if (q < n && !walks) S.srt[q] = (uint16_t)e;
        const unsigned m = __ballot_sync(0xffffffffu, walks);
        if (walks) S.p.walk[nwalk + __popc(m & ((1u << lane) - 1u))] = q | (e << 16);
        nwalk += __popc(m);
    }
}

// Step 1 by the keyed bijection (257 <= n <= 512): the eight round keys come from one Philox call
// in each of lanes 0-7; the round function of round r takes at most 32 distinct inputs (the other
// half, below A or B), so its values are tabulated once per cell in shared memory, and each
// position's image is eight table lookups, four positions per lane in flight.  The result is
// the same bijection as feistel(): L' = L + floor(h(R ^ Kx_r) A / 2^32) mod A, and likewise R.
template <typename SM>
__device__ __forceinline__ void warp_prp_list(const StepArgs& a, SM& S, uint32_t cell, uint32_t step, uint32_t n,
                                              uint32_t lane)
{
    const PrpDom dom = c_prp_dom.e[n - PRP_MIN_N];             // PRP_MIN_N <= n <= WC_MAX
    const uint32_t A = dom.ab & 0xffffu, B = dom.ab >> 16, Binv = dom.binv;
    {
        const U4 x = philox((lane >> 2) & 1u, cell, step, 2u, a.pk);
        const uint32_t K = u4_word(x, lane & 3u);
        const uint32_t Kx = K ^ (K >> 16);
#pragma unroll
        for (uint32_t r = 0; r < PRP_ROUNDS; ++r) {
            const uint32_t kr = __shfl_sync(0xffffffffu, Kx, r);
            const uint32_t M = (r & 1u) ? B : A, lim = (r & 1u) ? A : B;
            if (lane < lim) S.p.tab[r][lane] = (uint8_t)__umulhi(lowbias32_top16(lane ^ kr), M);
        }
    }
    __syncwarp();
    uint32_t nwalk = 0;
    for (uint32_t base = 0; base < n; base += 128) {          // 4, 2 or 1 positions per lane
        const uint32_t rest = n - base;
        if (rest > 64) prp_positions<4>(S, base, n, A, B, Binv, nwalk, lane);
        else if (rest > 32) prp_positions<2>(S, base, n, A, B, Binv, nwalk, lane);
        else prp_positions<1>(S, base, n, A, B, Binv, nwalk, lane);
    }
    __syncwarp();
    if (lane < nwalk) {                                        // nwalk < A <= 32: one lane each
        const uint32_t q = S.p.walk[lane] & 0xffffu;
        uint32_t e = S.p.walk[lane] >> 16;
        do {
            uint32_t h = __umulhi(e, Binv);
            if (h * B > e) --h;
            uint32_t Lw = h, Rw = e - h * B;
#pragma unroll
            for (uint32_t r = 0; r < PRP_ROUNDS; r += 2) {
                Lw = sub_mod(Lw + S.p.tab[r][Rw], A);
                Rw = sub_mod(Rw + S.p.tab[r + 1][Lw], B);
            }
            e = Lw * B + Rw;
        } while (e >= n);
        S.srt[q] = (uint16_t)e;
    }
}

// One cell's Steps 1-3 up to the early exit; the pairs it cannot settle are appended to the
// queue (WcQueue) for wc_pairs_kernel.
template <uint32_t SMAX>
__device__ void warp_cell_step(const StepArgs& a, const WcQueue& W, WarpCellSmem<SMAX>& S, uint32_t cell,
                               uint32_t step, LocalStats& ls, uint32_t lane)
{
    const uint64_t s0 = a.cell_start[cell];
    const uint32_t w = a.cell_start[cell + 1] - (uint32_t)s0;
    const uint32_t n = min(a.n_live[cell], w);
    if (n < 2) return;                                       // uniform
    const uint32_t kid = (uint32_t)a.kid[cell];
    const double dv = a.dv[cell];
    const float xup = __ull2float_ru(a.cell_xmax[cell]);     // no multiplicity of the cell is larger
    // the early exit's data of every SD: its volume bin, one byte (all of a lane's loads first)
    for (uint32_t base = 0; base < n; base += 256) {
        uint32_t b8[8];
#pragma unroll
        for (uint32_t k = 0; k < 8; ++k) {
            const uint32_t i = base + 32 * k + lane;
            b8[k] = i < n ? (uint32_t)__ldcs(a.vbin + s0 + i) : 0u;
        }
#pragma unroll
        for (uint32_t k = 0; k < 8; ++k) {
            const uint32_t i = base + 32 * k + lane;
            if (i < n) S.vb[i] = (uint8_t)b8[k];
        }
    }
    // Step 1: the shuffled list
    if (sorts(a, n)) {
        if (n > SMAX) {                                      // the host launches the SORT contract's
            if (lane == 0) atomicOr(a.err, ERR_TILE_OVERFLOW);   // instantiation: not reached
            return;
        }
        warp_sort_keys<SMAX>(a, S, cell, step, n, lane);
    } else {
        warp_prp_list(a, S, cell, step, n, lane);
    }
    __syncwarp();
    // Steps 2-3 up to the early exit: two pairs per lane and Philox call
    const float s32 = pair_ratio_dtdv_f(n, a.dt_f, dv);
    const float c_upx = __fmul_ru(exit_scale(s32, kid, a.golovin_bf, a.precision), xup);
    const float* __restrict__ tb = g_pbound[kid];
    const uint32_t npairs = n >> 1, G2 = (npairs + 1) >> 1;
    const uint32_t* __restrict__ srt2 = reinterpret_cast<const uint32_t*>(S.srt);   // pair m = srt2[m]
    for (uint32_t base = 0; base < G2; base += 32) {           // warp-uniform trip count
        const uint32_t M = base + lane;
        const bool valid = M < G2;
        U4 wv = {0, 0, 0, 0};
        if (valid) wv = philox(M, cell, step, 1u, a.pk);
        bool need[2];
        uint32_t ii[2];
#pragma unroll
        for (uint32_t h = 0; h < 2; ++h) {
            const uint32_t m = 2 * M + h;
            need[h] = false;
            ii[h] = 0;
            if (valid && m < npairs) {
                ii[h] = srt2[m];
                const float pup = __fmul_ru(__ldg(tb + pb_index(S.vb[ii[h] & 0xffffu], S.vb[ii[h] >> 16])), c_upx);
                need[h] = !(pup <= phi_lo23(h ? wv.z : wv.x));
                ls.pairs += need[h] ? 0u : 1u;
            }
        }
        // the lanes' surviving pairs go to the queue in one reservation per warp, lane by lane
        const unsigned m0 = __ballot_sync(0xffffffffu, need[0]), m1 = __ballot_sync(0xffffffffu, need[1]);
        const uint32_t tot = __popc(m0) + __popc(m1);
        if (tot) {
            uint32_t qb = 0;
            if (lane == 0) qb = atomicAdd(W.count, tot);
            const unsigned lt = (1u << lane) - 1u;
            qb = __shfl_sync(0xffffffffu, qb, 0) + __popc(m0 & lt) + __popc(m1 & lt);
#pragma unroll
            for (uint32_t h = 0; h < 2; ++h)
                if (need[h]) {
                    const uint64_t g1 = s0 + (ii[h] & 0xffffu), g2 = s0 + (ii[h] >> 16);
                    W.q[qb++] = make_uint4(cell, (uint32_t)g1, (uint32_t)g2, 2 * M + h);
                    // the pair kernel reads both SDs' multiplicities and volumes: this kernel
                    // leaves DRAM nearly idle, so start bringing them to L2 now
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(a.xi + g1));
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(a.xi + g2));
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(a.attr + g1));
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(a.attr + g2));
                }
        }
    }
}

// One warp per cell of at most 512 slots (see warp_cell_step).  SMAX: see WarpCellSmem (the SORT
// contract's instantiation sorts lists up to WC_MAX).
template <uint32_t SMAX>
__global__ void __launch_bounds__(32 * WC_WARPS, SMAX < WC_MAX ? SDM_WC_MIN_BLOCKS : 6) warp_cells_kernel(
    StepArgs a, WcQueue W, const uint32_t* __restrict__ cells, uint32_t n_cells)
{
    __shared__ WarpCellSmem<SMAX> ws[WC_WARPS];
    __shared__ unsigned long long red[8];
    // the pair kernel that follows may be scheduled as this grid drains (it waits for it to finish)
    asm volatile("griddepcontrol.launch_dependents;");
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t step = step_index(a);
    LocalStats ls = {0, 0, 0, 0, 0ull};
    if (threadIdx.x < 5) red[threadIdx.x] = 0;
    __syncthreads();
    for (uint32_t k = blockIdx.x * WC_WARPS + warp; k < n_cells; k += gridDim.x * WC_WARPS)
        warp_cell_step(a, W, ws[warp], cells[k], step, ls, lane);
    if (a.stats) {
        __syncthreads();
        flush_stats(a, ls, red);
    }
}

// The queued pairs of the small-cell step, one per thread (a warp takes 32 consecutive entries, so
// that the surrogate evaluates them together on the tensor cores): the pair's SDs and its cell's
// constants are gathered, then Step 2 and Step 3 (process_pair).  A cell that lost an SD is listed
// once for wc_compact_kernel.
template <bool SURR>
__global__ void __launch_bounds__(256, SURR ? 2 : 3) wc_pairs_kernel(StepArgs a, WcQueue W)
{
    __shared__ unsigned long long red[8];
    const EffTab* __restrict__ T = &g_eff_tab;
    if (threadIdx.x < 5) red[threadIdx.x] = 0;
    // launched as a programmatic dependent of the cell kernel: wait until its queue is complete
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    __syncthreads();
    LocalStats ls = {0, 0, 0, 0, 0ull};
    const uint32_t nq = *(volatile uint32_t*)W.count;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t step = step_index(a);
    for (uint32_t base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < nq; base += gridDim.x * blockDim.x) {
        const uint32_t e = base + lane;
        const bool act = e < nq;
        uint4 q = make_uint4(0, 0, 0, 0);
        if (act) q = __ldcs(W.q + e);
        const uint32_t cell = q.x;
        const uint64_t g1 = q.y, g2 = q.z;
        uint32_t n = 2, kid = 0;
        double dv = 1.0;
        if (act) {
            const uint32_t s0 = a.cell_start[cell];
            n = min(a.n_live[cell], a.cell_start[cell + 1] - s0);
            kid = (uint32_t)a.kid[cell];
            dv = a.dv[cell];
        }
        const double v1 = act ? a.attr[g1] : 0.0, v2 = act ? a.attr[g2] : 0.0;
        const uint64_t x1 = act ? a.xi[g1] : 1ull, x2 = act ? a.xi[g2] : 1ull;
        const CellCtx cc{cell, n, kid, pair_ratio_dtdv_f(n, a.dt_f, dv), dv};
        float Kh = SURR_PER_LANE;
        if (SURR && a.precision == PREC_SURROGATE)
            Kh = surr_pair_kernel_warp(a.surr, v1, v2, act && kid == 1);   // the warp's pairs on the tensor cores
        uint32_t rflag = 0;
        if (act) {
            const uint64_t u53 = phi_u53(a.pk, cell, step, q.w & ~WQ_BIG);
            process_pair<SURR>(a, T, cc, u53, g1, g2, x1, x2, v1, v2, ls, &rflag, Kh);
        }
        if (rflag && atomicExch(&W.flag[cell], 1u) == 0u) {
            if (q.w & WQ_BIG) W.bigcells[atomicAdd(W.count + 3, 1u)] = cell;
            else W.cells[atomicAdd(W.count + 1, 1u)] = cell;
        }
    }
    if (a.stats) {
        __syncthreads();
        flush_stats(a, ls, red);
    }
}

// Step 0 of the next step for the cells the queued pairs emptied slots of: each listed cell of
// one warp is compacted stably by one warp, each listed large cell by a whole block.  Resets the
// queue's counters and flags for the next step (the counts are read once, by every block, before
// any is cleared: the last block to take the ticket clears them).
__global__ void __launch_bounds__(256) wc_compact_kernel(StepArgs a, WcQueue W, uint32_t* ticket)
{
    __shared__ uint32_t wt[40];
    __shared__ uint32_t last;
    asm volatile("griddepcontrol.wait;" ::: "memory");      // the pair kernel has completed
    const uint32_t nc = *(volatile uint32_t*)(W.count + 1), nbg = *(volatile uint32_t*)(W.count + 3);
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < nc; k += (gridDim.x * blockDim.x) >> 5) {
        const uint32_t c = W.cells[k];
        const uint32_t s0 = a.cell_start[c], w = a.cell_start[c + 1] - s0;
        const uint32_t n_new = warp_compact_cell(a, s0, min(a.n_live[c], w), lane);
        if (lane == 0) {
            a.n_live[c] = n_new;
            W.flag[c] = 0;
        }
    }
    __syncthreads();
    for (uint32_t k = blockIdx.x; k < nbg; k += gridDim.x) {   // block-uniform
        const uint32_t c = W.bigcells[k];
        const uint32_t s0 = a.cell_start[c], w = a.cell_start[c + 1] - s0;
        const uint32_t n_new = block_compact_cell(a, s0, min(a.n_live[c], w), wt);
        if (threadIdx.x == 0) {
            a.n_live[c] = n_new;
            W.flag[c] = 0;
        }
        __syncthreads();
    }
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1 ? 1u : 0u;
    __syncthreads();
    if (last && threadIdx.x == 0) {
        W.count[0] = 0;
        W.count[1] = 0;
        W.count[3] = 0;
        *ticket = 0;
    }
}

// Per cell stepped by one warp: the largest multiplicity (an upper bound for the early exit of
// every later step until the state is replaced: coalescence never raises a multiplicity), and
// the volume bin of every slot.  One warp per cell of the list.
__global__ void cell_bounds_kernel(const uint64_t* __restrict__ xi, const double* __restrict__ vol,
                                   const uint32_t* __restrict__ cell_start, const uint32_t* __restrict__ cells,
                                   uint32_t n_cells, unsigned long long* __restrict__ xmax,
                                   uint8_t* __restrict__ vbin)
{
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n_cells; k += (gridDim.x * blockDim.x) >> 5) {
        const uint32_t c = cells[k];
        const uint32_t s0 = cell_start[c], s1 = cell_start[c + 1];
        unsigned long long m = 0;
        for (uint32_t i = s0 + lane; i < s1; i += 32) {
            m = max(m, (unsigned long long)xi[i]);
            vbin[i] = (uint8_t)vbin_of(vol[i]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) xmax[c] = m;
    }
}

// ---------------------------------------------------------------------------
// Large cells: bookkeeping shared by their kernels and the end-of-step
// compaction done by the last CTA of the step's final large-cell kernel.
// ---------------------------------------------------------------------------
struct BigBook {
    unsigned long long* ticket;   // SORT contract: low word: CTAs of the current kernel that
                                  // finished; high word: how many of them removed an SD
    uint32_t* removed;            // [n_big] an SD of this cell was removed during the step
    uint32_t n_big;
    uint32_t* sync;               // PRP contract, eight words (see big_prp_kernel):
                                  // [0], [1] some large cell awaits compaction, written by the
                                  //   launches of even and odd serial number respectively;
                                  // [2], [3] grid barrier count and generation;
                                  // [4..5] 64-bit arrival word: high half the serial number of
                                  //   the current launch, low half its CTAs that started
};
constexpr uint32_t BIG_SYNC_WORDS = 8;

constexpr uint32_t GRID_BARRIER_SPIN_LIMIT = 1u << 22;   // ~0.4 s of polling at >= 100 ns each

// Barrier of a cooperatively launched grid (every block resident).  Thread 0 of each block
// arrives on the counter; the last arrival resets it and advances the generation the others
// poll.  The poll gives up after spin_limit rounds: the error word gets ERR_TIMEOUT and false
// is returned (the caller then ends the kernel).
__device__ bool grid_barrier(uint32_t* count, uint32_t* gen, uint32_t* err,
                             uint32_t spin_limit = GRID_BARRIER_SPIN_LIMIT)
{
    __shared__ uint32_t ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t ok = 1;
        const uint32_t g = *(volatile uint32_t*)gen;              // read before arriving
        __threadfence();                                          // release this block's writes
        if (atomicAdd(count, 1u) == gridDim.x - 1) {
            *(volatile uint32_t*)count = 0;
            __threadfence();
            atomicExch(gen, g + 1u);
        } else {
            uint32_t it = 0;
            while (*(volatile uint32_t*)gen == g) {
                if (++it > spin_limit) {
                    atomicOr(err, ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();                                          // acquire the others' writes
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// Stable compaction of one cell by the whole block (chunks of blockDim slots;
// see warp_compact_cell).  wt needs 33 words of shared memory.
__device__ uint32_t block_compact_cell(const StepArgs& a, uint64_t base, uint32_t n_old, uint32_t* wt)
{
    const uint32_t tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t dst = 0;
    for (uint32_t r = 0; r <= a.n_attr; ++r) {
        dst = 0;
        for (uint32_t off = 0; off < n_old; off += nt) {
            const uint32_t i = off + tid;
            const bool in = i < n_old;
            const uint64_t x = in ? a.xi[base + i] : 0ull;
            const bool live = x != 0;
            const unsigned mask = __ballot_sync(0xffffffffu, live);
            if (lane == 0) wt[warp] = __popc(mask);
            __syncthreads();
            if (warp == 0) {
                const uint32_t w = lane < nw ? wt[lane] : 0u;
                uint32_t inc = w;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= (uint32_t)o) inc += t;
                }
                if (lane < nw) wt[lane] = inc - w;
                if (lane == 31) wt[32] = inc;
            }
            __syncthreads();
            const uint32_t pos = dst + wt[warp] + __popc(mask & lt);
            if (r < a.n_attr) {
                double* A = a.attr + (uint64_t)r * a.stride + base;
                const double v = in ? A[i] : 0.0;
                __syncthreads();
                if (live) {
                    A[pos] = v;
                    if (r == 0 && a.vbin) a.vbin[base + pos] = (uint8_t)vbin_of(v);
                }
            } else {
                __syncthreads();
                if (live) a.xi[base + pos] = x;
            }
            dst += wt[32];
            __syncthreads();
        }
    }
    for (uint32_t i = dst + tid; i < n_old; i += nt) {
        a.xi[base + i] = 0ull;
        for (uint32_t r = 0; r < a.n_attr; ++r) a.attr[(uint64_t)r * a.stride + base + i] = 0.0;
        if (a.vbin) a.vbin[base + i] = 0;
    }
    __syncthreads();
    return dst;
}

// Called by every CTA at its end (had_removal: some thread of the CTA removed an
// SD): the last CTA compacts the large cells that lost SDs in this step and
// resets the bookkeeping.  One atomic per CTA; the removal count travels in the
// same word, so without removals the last CTA reads nothing else.
__device__ void big_end_of_step(const StepArgs& a, const BigCell* __restrict__ cells, const BigBook& bk, uint32_t* wt,
                                bool had_removal)
{
    __shared__ unsigned long long s_old;
    const bool any = __syncthreads_or(had_removal);
    if (threadIdx.x == 0) {
        // release: this CTA's updates (ordered before by the barrier) become visible to the
        // CTA that sees the last ticket; acquire: that CTA sees everybody's
        unsigned long long old;
        const unsigned long long inc = 1ull + (any ? (1ull << 32) : 0ull);
        asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(bk.ticket), "l"(inc) : "memory");
        s_old = old;
    }
    __syncthreads();
    const unsigned long long old = s_old;
    if ((uint32_t)old != gridDim.x - 1) return;
    if (threadIdx.x == 0) *bk.ticket = 0ull;
    if ((old >> 32) == 0 && !any) return;
    __threadfence();
    for (uint32_t b = 0; b < bk.n_big; ++b) {
        if (!*(volatile uint32_t*)&bk.removed[b]) continue;
        const BigCell C = cells[b];
        const uint32_t n_old = min(*(volatile uint32_t*)&a.n_live[C.cell], C.width);
        const uint32_t n_new = block_compact_cell(a, C.slot_begin, n_old, wt);
        if (threadIdx.x == 0) {
            a.n_live[C.cell] = n_new;
            bk.removed[b] = 0;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Large cells under the PRP contract.  The candidate pairs of all large cells
// are taken two at a time -- a "quad": list positions 4q .. 4q+3, pairs 2q and
// 2q+1, whose phi come from one Philox call -- and the quads, numbered across
// the cells (BigCell::quad_begin), are split into equal contiguous ranges, one
// per CTA of a single-wave grid.  Every thread derives the cell's round keys
// itself (no shared context, no barrier before work starts) and takes two
// quads at a time: it maps their eight positions through the keyed bijection,
// issues all eight gathers, computes phi while they are in flight, and settles
// most pairs by the early exit (phi above an upper bound of p).  The remaining
// pairs go to a per-warp queue in shared memory and are evaluated 32 at a
// time, so the long evaluation runs on full warps instead of diverging the
// common path.
// ---------------------------------------------------------------------------
constexpr uint32_t PRP_THREADS = 128;           // threads per CTA (one or a few large cells)
constexpr uint32_t PRP_THREADS_MANY = 64;       // threads per CTA with many large cells: finer ranges
constexpr uint32_t PRP_MANY_CELLS = 64;         // large cells from which the finer CTAs are used
constexpr uint32_t PRP_WARPS = PRP_THREADS / 32;
#ifndef SDM_PRP_MIN_BLOCKS
#define SDM_PRP_MIN_BLOCKS 4
#endif
#ifndef SDM_PRP_QPT
#define SDM_PRP_QPT 4
#endif
constexpr uint32_t PRP_QPT = SDM_PRP_QPT;      // quads per thread and iteration
constexpr uint32_t BIG_PARAM_CELLS = 8;        // large cells passed by value in the launch
constexpr uint32_t PQ_CAP = 2 * 32 * PRP_QPT;   // queued pairs per warp (2 per quad; emptied every iteration)

struct BigLaunch {
    uint32_t n_big, n_quads;
    const BigCell* cells;                      // [n_big] (device)
    const unsigned long long* xmax;            // [n_big] largest multiplicity of the cell (since the upload)
    const uint32_t* cta_first;                 // [grid] first large cell of each CTA (n_big > BIG_PARAM_CELLS)
    BigCell pc[BIG_PARAM_CELLS];               // the large cells when n_big <= BIG_PARAM_CELLS
};

struct PairQueue {
    uint32_t s1[PQ_CAP], s2[PQ_CAP];
    unsigned long long u[PQ_CAP];
};

// N Feistel evaluations with shared round keys (independent chains).  The rounds
// are a loop with the keys rotated through registers, not unrolled: with the
// state flushed from L2 before every step the instructions are fetched from
// DRAM each time, and straight-line code of all rounds stalls on the fetch.
// N images through the network.  FULL: the domain is a power of two (A = 2^a,
// B = 2^b), where floor(h M / 2^32) is a shift and the modulo a mask; otherwise
// the general form (a multiply-high and a conditional subtraction).  Both forms
// compute the same network on a power-of-two domain.
template <int N, bool FULL>
__device__ __forceinline__ void feistel_n(const Prp& P, uint32_t (&x)[N])
{
    uint32_t L[N], R[N];
    uint32_t k0 = P.K[0], k1 = P.K[1], k2 = P.K[2], k3 = P.K[3], k4 = P.K[4], k5 = P.K[5], k6 = P.K[6],
             k7 = P.K[7];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (FULL) { L[i] = x[i] >> P.b; R[i] = x[i] & (P.B - 1u); }
        else prp_split(P, x[i], L[i], R[i]);
    }
#pragma unroll 1
    for (uint32_t r = 0; r < PRP_ROUNDS; r += 2) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            if (FULL) prp_round_pair_pow2(P, k0, k1, L[i], R[i]);
            else prp_round_pair(P, k0, k1, L[i], R[i]);
        }
        k0 = k2; k1 = k3; k2 = k4; k3 = k5; k4 = k6; k5 = k7;
    }
#pragma unroll
    for (int i = 0; i < N; ++i)
        x[i] = FULL ? (((L[i] & (P.A - 1u)) << P.b) | (R[i] & (P.B - 1u))) : L[i] * P.B + R[i];
}

// Cycle-walking of a warp's images by a work list instead of per-lane loops.
// An image outside [0, n) goes through the network again until it lands inside;
// the network's domain holds fewer than n + sqrt(n) + 1 elements, so few images
// walk, but a per-lane loop would still keep the whole warp busy for the
// longest walk of any of its 32 x N images.  Here the images still walking are compacted into a list
// in shared memory and advanced WALK_ILP per lane per pass, so every pass runs
// on full lanes.  The results are the same images the per-lane loop gives.
constexpr int WALK_ILP = 4;
struct WalkScratch {                       // per warp, two lists of (value, owner) used alternately
    uint32_t val[2][256], res[256];
    uint8_t tag[2][256];
};

template <int N>
__device__ __forceinline__ void prp_walk_list(const Prp& P, uint32_t use, uint32_t (&e)[N], WalkScratch& W,
                                              uint32_t lane)
{
    static_assert(32 * N <= 256, "walk list too small");
    uint32_t mine = 0;                     // images of this lane still outside [0, n)
#pragma unroll
    for (int i = 0; i < N; ++i) mine |= (((use >> i) & 1u) && e[i] >= P.n) ? (1u << i) : 0u;
    if (!__any_sync(0xffffffffu, mine != 0)) return;
    // list the walking images (owner = lane * N + i)
    uint32_t cnt = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const bool w = (mine >> i) & 1u;
        const unsigned m = __ballot_sync(0xffffffffu, w);
        if (w) {
            const uint32_t k = cnt + __popc(m & ((1u << lane) - 1u));
            W.val[0][k] = e[i];
            W.tag[0][k] = lane * N + i;
        }
        cnt += __popc(m);
    }
    uint32_t cur = 0;
    for (uint32_t pass = 0; cnt > 0 && pass < 4096; ++pass) {   // each pass strictly shrinks or keeps the list
        __syncwarp();
        uint32_t x[WALK_ILP], t[WALK_ILP];
        bool have[WALK_ILP];
#pragma unroll
        for (int w = 0; w < WALK_ILP; ++w) {
            const uint32_t k = lane + 32 * w;
            have[w] = k < cnt;
            x[w] = have[w] ? W.val[cur][k] : 0u;
            t[w] = have[w] ? W.tag[cur][k] : 0u;
        }
        feistel_n<WALK_ILP, false>(P, x);
        uint32_t nxt = 0;
#pragma unroll
        for (int w = 0; w < WALK_ILP; ++w) {
            const bool again = have[w] && x[w] >= P.n;
            if (have[w] && !again) W.res[t[w]] = x[w];
            const unsigned m = __ballot_sync(0xffffffffu, again);
            if (again) {
                const uint32_t k = nxt + __popc(m & ((1u << lane) - 1u));
                W.val[cur ^ 1][k] = x[w];
                W.tag[cur ^ 1][k] = t[w];
            }
            nxt += __popc(m);
        }
        // entries beyond 32 * WALK_ILP were not taken this pass: carry them over unchanged
        for (uint32_t k = 32 * WALK_ILP + lane; k < cnt; k += 32) {
            // appended after this pass's re-queued images (order does not matter)
            const uint32_t dst = nxt + (k - 32 * WALK_ILP);
            W.val[cur ^ 1][dst] = W.val[cur][k];
            W.tag[cur ^ 1][dst] = W.tag[cur][k];
        }
        if (cnt > 32 * WALK_ILP) nxt += cnt - 32 * WALK_ILP;
        cnt = nxt;
        cur ^= 1;
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < N; ++i)
        if ((mine >> i) & 1u) e[i] = W.res[lane * N + i];
    __syncwarp();
}

// Evaluate the top 'take' queued pairs of this warp (lanes < take) and pop them.
template <bool SURR>
__device__ __forceinline__ void drain_queue(const StepArgs& a, const EffTab* __restrict__ T, const CellCtx& cc,
                                            PairQueue& Q, uint32_t& qcnt, uint32_t take, LocalStats& ls,
                                            uint32_t* removed_flag, uint32_t lane)
{
    __syncwarp();
    const bool act = lane < take;
    const uint32_t k = qcnt - take + lane;
    const uint32_t s1 = act ? Q.s1[k] : 0u, s2 = act ? Q.s2[k] : 0u;
    const double v1 = act ? a.attr[s1] : 0.0, v2 = act ? a.attr[s2] : 0.0;
    float Kh = SURR_PER_LANE;
    if (SURR && a.precision == PREC_SURROGATE && cc.kid == 1)
        Kh = surr_pair_kernel_warp(a.surr, v1, v2, act);         // the warp's pairs on the tensor cores
    if (act) process_pair<SURR>(a, T, cc, Q.u[k], s1, s2, a.xi[s1], a.xi[s2], v1, v2, ls, removed_flag, Kh);
    __syncwarp();
    qcnt -= take;
}

// Settle pair (s1, s2) by the early exit or queue it (warp-collective).  k1, k2 are
// the volumes' bins (vbin_of); c_upx is the cell's early-exit scale times its
// multiplicity bound.
__device__ __forceinline__ void exit_or_queue(const StepArgs& a, PairQueue& Q, uint32_t& qcnt, bool has, uint32_t s1,
                                              uint32_t s2, uint32_t k1, uint32_t k2, uint32_t w_hi, uint32_t w_lo,
                                              const float* __restrict__ tb, float c_upx, LocalStats& ls,
                                              uint32_t lane)
{
    bool need = false;
    if (has) {
        need = !(__fmul_ru(__ldg(tb + pb_index(k1, k2)), c_upx) <= phi_lo23(w_hi));
        ls.pairs += need ? 0u : 1u;
    }
    const unsigned m = __ballot_sync(0xffffffffu, need);
    if (need) {
        const uint32_t k = qcnt + __popc(m & ((1u << lane) - 1u));
        Q.s1[k] = s1;
        Q.s2[k] = s2;
        Q.u[k] = ((((uint64_t)w_hi) << 32) | (uint64_t)w_lo) >> 11;
        // the multiplicities are read when the queue is drained: start bringing them to L2
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a.xi + s1));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a.xi + s2));
    }
    qcnt += __popc(m);
}

// The same for a layout whose large cells' surviving pairs go to the step's queue (evaluated by
// wc_pairs_kernel, the cells that lost SDs compacted by wc_compact_kernel): (cell, slots, pair
// index m | WQ_BIG) appended, one reservation per warp; the SDs' multiplicities and volumes
// prefetched into L2 for the pair kernel.
__device__ __forceinline__ void exit_or_gqueue(const StepArgs& a, const WcQueue& W, bool has, uint32_t cell,
                                               uint32_t s1, uint32_t s2, uint32_t m, uint32_t k1, uint32_t k2,
                                               uint32_t w_hi, const float* __restrict__ tb, float c_upx,
                                               LocalStats& ls, uint32_t lane)
{
    bool need = false;
    if (has) {
        need = !(__fmul_ru(__ldg(tb + pb_index(k1, k2)), c_upx) <= phi_lo23(w_hi));
        ls.pairs += need ? 0u : 1u;
    }
    const unsigned mk = __ballot_sync(0xffffffffu, need);
    if (mk) {
        uint32_t qb = 0;
        if (lane == 0) qb = atomicAdd(W.count, (uint32_t)__popc(mk));
        qb = __shfl_sync(0xffffffffu, qb, 0) + __popc(mk & ((1u << lane) - 1u));
        if (need) {
            W.q[qb] = make_uint4(cell, s1, s2, m | WQ_BIG);
            asm volatile("prefetch.global.L2 [%0];" ::"l"(a.xi + s1));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(a.xi + s2));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(a.attr + s1));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(a.attr + s2));
        }
    }
}

// The quads [sa, sb) of one large cell for one warp: per iteration PRP_QPT quads
// per lane (quads g, g + 32, ...; a warp-uniform trip count), their bijection
// images, the gathers of the volumes' high words, the early exit and the queue
// of pairs that need the kernel.  FULL: n = A B is a power of two, so no image
// walks and the rounds take their shift-and-mask form.  GQ: the surviving pairs go to the step's
// queue W instead of the warp's (whose memory then only holds the walk lists).
template <bool SURR, bool FULL, bool GQ>
__device__ __forceinline__ void prp_cell_quads(const StepArgs& a, const EffTab* __restrict__ tab, const CellCtx& cc,
                                               const Prp& P, const BigCell& C, uint32_t sa, uint32_t sb,
                                               uint32_t step, const float* __restrict__ tb, float c_upx, PairQueue& Q,
                                               uint32_t& qcnt, LocalStats& ls, uint32_t* rflag, uint32_t warp,
                                               uint32_t lane, uint32_t nt, const WcQueue& W)
{
    const uint32_t npairs = cc.n >> 1;
    // PRP_QPT quads per thread and iteration: g, g + 32, ... (warp-uniform trip count)
    constexpr int NP = 4 * PRP_QPT;            // positions per thread and iteration
    for (uint32_t base = sa + warp * 32 * PRP_QPT; base < sb; base += PRP_QPT * nt) {
        uint32_t e[NP], qj[PRP_QPT];
#pragma unroll
        for (int j = 0; j < (int)PRP_QPT; ++j) {
            qj[j] = base + 32 * j + lane - C.quad_begin;
#pragma unroll
            for (int i = 0; i < 4; ++i) e[4 * j + i] = 4 * qj[j] + i;
        }
        bool h0[PRP_QPT], h1[PRP_QPT];
        uint32_t use = 0;
#pragma unroll
        for (int j = 0; j < (int)PRP_QPT; ++j) {
            h0[j] = base + 32 * j + lane < sb && 2 * qj[j] < npairs;
            h1[j] = h0[j] && 2 * qj[j] + 1 < npairs;
            use |= (h0[j] ? 3u : 0u) << (4 * j);
            use |= (h1[j] ? 12u : 0u) << (4 * j);
        }
        // Two halves: the second half's bijection images are computed while the first
        // half's gathers are in flight.  Only the volumes' bins are gathered (1 byte per
        // SD from the bin array, else the volume's high word): with the cell's
        // multiplicity bound they are all the early exit needs.
        constexpr int NH = NP / 2;
        uint32_t vh[NP];
        const uint32_t* attr_hi = reinterpret_cast<const uint32_t*>(a.attr) + 1;
        const uint8_t* __restrict__ vbin = a.vbin;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            uint32_t eh[NH];
#pragma unroll
            for (int i = 0; i < NH; ++i) eh[i] = e[NH * hh + i];
            feistel_n<NH, FULL>(P, eh);
            // the pair queue is empty here: its memory holds the walk list
            if (!FULL) prp_walk_list<NH>(P, use >> (NH * hh), eh, *reinterpret_cast<WalkScratch*>(&Q), lane);
#pragma unroll
            for (int i = 0; i < NH; ++i) {
                e[NH * hh + i] = eh[i] + C.slot_begin;   // slots from here on
                const uint32_t ei = e[NH * hh + i];
                vh[NH * hh + i] = !((use >> (NH * hh + i)) & 1u) ? 0u
                                  : vbin ? (uint32_t)vbin[ei] : pb_bin_key(attr_hi[2 * (size_t)ei] >> 18);
            }
        }
        // phi while the gathers are in flight, then the early exit
#pragma unroll
        for (int j = 0; j < (int)PRP_QPT; ++j) {
            U4 w = {0, 0, 0, 0};
            if (h0[j]) w = philox(qj[j], C.cell, step, 1u, a.pk);
            if (GQ) {
                exit_or_gqueue(a, W, h0[j], C.cell, e[4 * j], e[4 * j + 1], 2 * qj[j], vh[4 * j], vh[4 * j + 1], w.x,
                               tb, c_upx, ls, lane);
                exit_or_gqueue(a, W, h1[j], C.cell, e[4 * j + 2], e[4 * j + 3], 2 * qj[j] + 1, vh[4 * j + 2],
                               vh[4 * j + 3], w.z, tb, c_upx, ls, lane);
            } else {
                exit_or_queue(a, Q, qcnt, h0[j], e[4 * j], e[4 * j + 1], vh[4 * j], vh[4 * j + 1], w.x, w.y, tb,
                              c_upx, ls, lane);
                exit_or_queue(a, Q, qcnt, h1[j], e[4 * j + 2], e[4 * j + 3], vh[4 * j + 2], vh[4 * j + 3], w.z,
                              w.w, tb, c_upx, ls, lane);
            }
        }
        if (GQ) {
        } else if (FULL) {
            while (qcnt >= 32) drain_queue<SURR>(a, tab, cc, Q, qcnt, 32, ls, rflag, lane);
        } else {                      // empty the queue for the next walk list
            while (qcnt > 0) drain_queue<SURR>(a, tab, cc, Q, qcnt, min(qcnt, 32u), ls, rflag, lane);
        }
    }
    if (!GQ && qcnt > 0) drain_queue<SURR>(a, tab, cc, Q, qcnt, qcnt, ls, rflag, lane);
}

// THREADS: CTA size (the same registers and warps per SM for both sizes)
// STEP0: the launch may find cells flagged by the previous launch and compact them first (the
// allocating path); false where a compaction kernel always follows the step (the
// allocation-free call, and GQ), so no launch ever starts with a flagged cell.
// GQ: the surviving pairs go to the step's queue W (wc_pairs_kernel decides them and
// wc_compact_kernel compacts the cells that lost SDs, in the same step): the kernel then holds
// neither the pairs' decisions nor Step 0.
template <bool SURR, uint32_t THREADS = PRP_THREADS, bool STEP0 = true, bool GQ = false>
__global__ void __launch_bounds__(THREADS, (GQ ? 3 : 2) * SDM_PRP_MIN_BLOCKS * PRP_THREADS / THREADS / 2)
    big_prp_kernel(StepArgs a, BigLaunch L, BigBook bk, WcQueue W)
{
    const EffTab* __restrict__ tab = &g_eff_tab;   // read through L1: no staging on the critical path
    // a compaction kernel that follows (allocation-free step) may start launching
    asm volatile("griddepcontrol.launch_dependents;");
    __shared__ PairQueue pq[THREADS / 32];
    __shared__ uint32_t wt[40];
    static_assert(sizeof(WalkScratch) <= sizeof(PairQueue), "the walk list shares the pair queue's memory");
    __shared__ uint32_t key_s[PRP_MIN_N];
    __shared__ uint16_t srt_s[PRP_MIN_N];
    __shared__ unsigned long long red[8];
    const uint32_t tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t step = step_index(a);
    const uint32_t qa = (uint32_t)(((uint64_t)blockIdx.x * L.n_quads) / gridDim.x);
    const uint32_t qb = (uint32_t)(((uint64_t)(blockIdx.x + 1) * L.n_quads) / gridDim.x);
    const bool by_value = L.n_big <= BIG_PARAM_CELLS;
    uint32_t c = 0;                                 // first large cell of this CTA's range
    if (by_value) {
        for (uint32_t k = 1; k < L.n_big; ++k)
            if (L.pc[k].quad_begin <= qa) c = k;
    } else {
        c = L.cta_first[blockIdx.x];
    }
    LocalStats ls = {0, 0, 0, 0, 0ull};
    if (tid < 5) red[tid] = 0;
    // the bound table (read right after the gathers) and the efficiency table (read by the
    // queued evaluations) are cold after other work evicted L2: start fetching them now --
    // the bound table into L2, a slice per CTA, the efficiency table into every SM's L1
    {
        constexpr uint32_t PB_LINES = (uint32_t)((sizeof(g_pbound) + 127) / 128);
        for (uint32_t l = blockIdx.x * nt + tid; l < PB_LINES; l += gridDim.x * nt)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char*>(g_pbound) + 128 * l));
        constexpr uint32_t EFF_LINES = (uint32_t)((sizeof(EffTab) + 127) / 128);
        static_assert(EFF_LINES <= 32, "one line per lane");
        if (warp == 0 && lane < EFF_LINES)
            asm volatile("prefetch.global.L1 [%0];" ::"l"(reinterpret_cast<const char*>(tab) + 128 * lane));
        // the second filter's FP64 tables, into L2 (a few pairs per step read them)
        constexpr uint32_t ED_LINES = (uint32_t)((sizeof(g_eff_Ed) + 127) / 128);
        static_assert(ED_LINES + 2 <= 32, "one line per lane");
        if (blockIdx.x == 0 && warp == 1) {
            const char* line = lane < ED_LINES ? reinterpret_cast<const char*>(g_eff_Ed) + 128 * lane
                               : lane == ED_LINES  ? reinterpret_cast<const char*>(g_eff_Rd)
                                                   : reinterpret_cast<const char*>(g_eff_invdRd);
            if (lane < ED_LINES + 2) asm volatile("prefetch.global.L2 [%0];" ::"l"(line));
        }
    }
    // Step 0 for the large cells that lost SDs in the previous launch: each such cell is compacted
    // by one block while the grid waits at a barrier (the launch is cooperative).  CTAs of this
    // launch may finish, and flag their cells, before other CTAs of it have started, so the
    // pending word a launch reads is never one it writes: launch number k (taken from the arrival
    // word: every CTA adds one, the last to arrive moves the count into the serial number) reads
    // the word of parity k+1, written by launch k-1, and writes the word of parity k.  Nobody
    // writes the word it reads before every CTA has passed the barrier; then block 0 clears it.
    __shared__ uint32_t par_s, pend_s;
    uint32_t par = 0;
    if (STEP0) {
        if (tid == 0) {
            const uint32_t p0 = __ldcg(bk.sync), p1 = __ldcg(bk.sync + 1);
            unsigned long long* arr = reinterpret_cast<unsigned long long*>(bk.sync + 4);
            const unsigned long long old = atomicAdd(arr, 1ull);
            if ((uint32_t)old == gridDim.x - 1u) atomicAdd(arr, (1ull << 32) - gridDim.x);
            const uint32_t k = (uint32_t)(old >> 32) & 1u;
            par_s = k;
            pend_s = k ? p0 : p1;
        }
        __syncthreads();
        par = par_s;
        if (pend_s != 0u) {
            for (uint32_t b = blockIdx.x; b < L.n_big; b += gridDim.x) {
                if (!__ldcg(&bk.removed[b])) continue;
                const BigCell C = L.cells[b];
                const uint32_t n_old = min(__ldcg(&a.n_live[C.cell]), C.width);
                const uint32_t n_new = block_compact_cell(a, C.slot_begin, n_old, wt);
                if (tid == 0) {
                    a.n_live[C.cell] = n_new;
                    bk.removed[b] = 0;
                }
            }
            if (!grid_barrier(bk.sync + 2, bk.sync + 3, a.err)) return;
            if (blockIdx.x == 0 && tid == 0) *(volatile uint32_t*)(bk.sync + (par ^ 1u)) = 0u;
        }
    }
    PairQueue& Q = pq[warp];
    uint32_t qcnt = 0;                              // queued pairs of this warp (warp-uniform)
    for (; qa < qb && c < L.n_big; ++c) {
        const BigCell C = by_value ? L.pc[c] : L.cells[c];
        if (C.quad_begin >= qb) break;
        const uint32_t q_end = c + 1 < L.n_big ? (by_value ? L.pc[c + 1].quad_begin : L.cells[c + 1].quad_begin)
                                               : L.n_quads;
        const uint32_t sa = max(qa, C.quad_begin), sb = min(qb, q_end);
        // the cell's context, in every thread; the round keys are derived while the live
        // count n is loading
        const uint32_t n = min(__ldcg(&a.n_live[C.cell]), C.width);
        const uint32_t kid = (uint32_t)a.kid[C.cell];
        const double dv = a.dv[C.cell];
        const float xup = __ull2float_ru(L.xmax[c]);
        Prp P;
        prp_init(P, a.pk, C.cell, step, C.width);
        const float* __restrict__ tb = g_pbound[kid];
        uint32_t* const rflag = &bk.removed[c];
        const uint32_t npairs = n >> 1;
        if (n >= PRP_MIN_N) {
            const float s32 = pair_ratio_dtdv_f(n, a.dt_f, dv);
            const CellCtx cc{C.cell, n, kid, s32, dv};
            const float c_upx = __fmul_ru(exit_scale(s32, kid, a.golovin_bf, a.precision), xup);
            if (P.pow2 && n == C.width) {
                prp_cell_quads<SURR, true, GQ>(a, tab, cc, P, C, sa, sb, step, tb, c_upx, Q, qcnt, ls, rflag, warp,
                                               lane, nt, W);
            } else {
                if (!prp_same_network(P, n)) prp_set_domain(P, n);
                P.n = n;
                prp_cell_quads<SURR, false, GQ>(a, tab, cc, P, C, sa, sb, step, tb, c_upx, Q, qcnt, ls, rflag, warp,
                                                lane, nt, W);
            }
        } else if (n >= 2 && C.quad_begin >= qa) {
            // few live SDs left in a large cell: sorted by key by the CTA holding the cell's
            // first quad (n, qa and the cell are the same in all threads: a uniform branch)
            __syncthreads();
            for (uint32_t t = tid; t < n; t += nt)
                key_s[t] = u4_word(philox(t >> 2, C.cell, step, 0u, a.pk), t & 3u);
            __syncthreads();
            for (uint32_t t = tid; t < n; t += nt) {
                const uint32_t kt = key_s[t];
                uint32_t r = 0;
                for (uint32_t j = 0; j < n; ++j) r += (key_s[j] < kt) || (key_s[j] == kt && j < t);
                srt_s[r] = (uint16_t)t;
            }
            __syncthreads();
            if (GQ) {                                   // every pair to the step's queue
                for (uint32_t m0 = warp * 32; m0 < npairs; m0 += nt) {   // warp-uniform
                    const uint32_t mm = m0 + lane;
                    const unsigned mk = __ballot_sync(0xffffffffu, mm < npairs);
                    uint32_t qb = 0;
                    if (lane == 0) qb = atomicAdd(W.count, (uint32_t)__popc(mk));
                    qb = __shfl_sync(0xffffffffu, qb, 0) + lane;
                    if (mm < npairs)
                        W.q[qb] = make_uint4(C.cell, C.slot_begin + srt_s[2 * mm], C.slot_begin + srt_s[2 * mm + 1],
                                             mm | WQ_BIG);
                }
            } else {
                const CellCtx cc{C.cell, n, kid, pair_ratio_dtdv_f(n, a.dt_f, dv), dv};
                for (uint32_t mm = tid; mm < npairs; mm += nt) {
                    const uint64_t s1 = C.slot_begin + srt_s[2 * mm], s2 = C.slot_begin + srt_s[2 * mm + 1];
                    process_pair<SURR>(a, tab, cc, phi_u53(a.pk, C.cell, step, mm), s1, s2, a.xi[s1],
                                 a.xi[s2], a.attr[s1], a.attr[s2], ls, rflag);
                }
            }
        }
    }
    if (a.stats) {
        __syncthreads();
        flush_stats(a, ls, red);
    }
    // cells that lost SDs are compacted at the start of the next launch (or by big_compact_kernel)
    if (__any_sync(0xffffffffu, ls.removed != 0) && lane == 0) atomicOr(bk.sync + par, 1u);
}

// Step 0 for the large cells of the PRP contract outside a PRP step: compacts,
// stably, the cells flagged by the last step and resets the flags -- before the
// state is read or stepped under the SORT contract, and after every
// allocation-free step.  There it is launched as a programmatic dependent: its
// blocks may be scheduled while the step's last blocks finish, and
// griddepcontrol.wait returns once the step grid has completed and its memory
// operations are visible.  After a plain launch the wait returns at once and
// stream order gives the same guarantee.
__global__ void __launch_bounds__(256) big_compact_kernel(StepArgs a, const BigCell* __restrict__ cells,
                                                          uint32_t* removed, uint32_t n_big, uint32_t* sync)
{
    __shared__ uint32_t wt[40];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (blockIdx.x == 0 && threadIdx.x == 0) sync[0] = sync[1] = 0u;   // every flagged cell is handled below
    for (uint32_t b = blockIdx.x; b < n_big; b += gridDim.x) {
        const uint32_t flag = *(volatile uint32_t*)&removed[b];   // the same in every thread
        if (!flag) continue;
        const BigCell C = cells[b];
        const uint32_t n_old = min(a.n_live[C.cell], C.width);
        const uint32_t n_new = block_compact_cell(a, C.slot_begin, n_old, wt);
        __syncthreads();
        if (threadIdx.x == 0) {
            a.n_live[C.cell] = n_new;
            removed[b] = 0;
        }
    }
}

// Self-test of the bounded wait: the grid meets at grid_barrier with the given spin limit;
// with withhold set, the last block never arrives (returns at once), so the others' wait runs
// out, they record ERR_TIMEOUT and return.  Launched cooperatively with a few blocks.
__global__ void barrier_selftest_kernel(uint32_t* count, uint32_t* gen, uint32_t* err, uint32_t spin_limit,
                                        uint32_t withhold)
{
    if (withhold && blockIdx.x == gridDim.x - 1) return;
    grid_barrier(count, gen, err, spin_limit);
}

// ---------------------------------------------------------------------------
// Large cells, pass 1: scatter (key, position) into fixed-capacity buckets.
// ---------------------------------------------------------------------------
constexpr uint32_t BIG_CHUNK = 2048;          // slots per scatter CTA (multiple of 4)
constexpr uint32_t BIG_SCATTER_THREADS = 256;
constexpr uint32_t BIG_GROUPS_PER_THREAD = BIG_CHUNK / 4 / BIG_SCATTER_THREADS;
constexpr uint32_t BIG_MAX_BUCKET_BITS = 13;  // <= 8192 buckets per cell
constexpr uint32_t BIG_ATOMIC_ILP = 4;        // bucket reservations in flight per thread

// Bucket bookkeeping shared by the two passes.
//   cursor[g]        records appended to bucket g in this step (zero between steps)
//   ticket[c]        scatter CTAs of large cell c that finished (zero between steps)
//   plan[g]          for bucket g: (start of the bucket in its cell's sorted list, its
//                    capacity-clamped record count, the cell's total, 0); the total is
//                    BUCKET_OVERFLOWED in every bucket of a cell when one of its buckets
//                    received more records than its capacity (the finishing pass then leaves
//                    the cell unchanged).  Written by the last scatter CTA of the cell, which
//                    also clears the cell's cursors and ticket.
constexpr uint32_t BUCKET_OVERFLOWED = 0xffffffffu;
struct BucketBook {
    uint32_t* cursor;
    uint4* plan;
    uint32_t* ticket;
    uint32_t n_buckets;
    uint32_t cap;
};

// The last scatter CTA of a cell: the plan of its nb buckets (nb a power of two, at most
// 8192; blockDim.x == BIG_SCATTER_THREADS).  Each thread takes nb / 256 consecutive
// buckets (at least one), loading them sixteen at a time with all sixteen loads in flight
// (so 4096 buckets cost one round trip to L2), staging the clamped counts in
// shared memory tmp[nb]; then a block scan of the thread sums.
__device__ void cell_bucket_plan(uint32_t* __restrict__ cursor, uint4* __restrict__ plan, uint32_t nb,
                                 uint32_t cap, uint32_t* tmp, uint32_t* wt, uint32_t* err)
{
    constexpr uint32_t BATCH = 16;
    const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const uint32_t per = nb > BIG_SCATTER_THREADS ? nb / BIG_SCATTER_THREADS : 1u;
    const uint32_t b0 = tid * per, b1 = min(nb, b0 + per);
    uint32_t over = 0, s = 0;
    for (uint32_t j0 = b0; j0 < b1; j0 += BATCH) {
        uint32_t v[BATCH];
#pragma unroll
        for (uint32_t j = 0; j < BATCH; ++j) v[j] = j0 + j < b1 ? __ldcg(&cursor[j0 + j]) : 0u;
#pragma unroll
        for (uint32_t j = 0; j < BATCH; ++j) {
            if (j0 + j < b1) {
                cursor[j0 + j] = 0u;
                over |= v[j] > cap;
                tmp[j0 + j] = min(v[j], cap);
                s += min(v[j], cap);
            }
        }
    }
    if (over) atomicOr(err, ERR_BUCKET_OVERFLOW);
    const bool cell_over = __syncthreads_or(over) != 0;
    uint32_t inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= (uint32_t)o) inc += t;
    }
    if (lane == 31) wt[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const uint32_t nw = BIG_SCATTER_THREADS / 32;
        const uint32_t w = lane < nw ? wt[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= (uint32_t)o) wi += t;
        }
        if (lane < nw) wt[lane] = wi - w;
        if (lane == 31) wt[32] = cell_over ? BUCKET_OVERFLOWED : wi;   // the cell's total
    }
    __syncthreads();
    const uint32_t total = wt[32];
    uint32_t run = wt[wid] + inc - s;
    for (uint32_t j = b0; j < b1; ++j) {
        const uint32_t c = tmp[j];
        plan[j] = make_uint4(run, c, total, 0u);
        run += c;
    }
}

// Records of bucket b (capacity cap) live at rec + b * cap, one 8-byte word
// each: (key << 32) | position in the cell's live list.  The live SDs of a cell
// are the prefix [0, n_live) of its slots (Step 0 ran before), so the pass reads
// no SD data at all: the keys come from the counter-based generator, the bucket
// is the key's top bits.  The finishing pass gathers what it needs per pair.
__global__ void __launch_bounds__(BIG_SCATTER_THREADS) big_scatter_kernel(StepArgs a, const BigCell* __restrict__ cells,
                                                                         const BigChunk* __restrict__ chunks,
                                                                         uint64_t* __restrict__ rec, BucketBook bk)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_last;
    __shared__ uint32_t wt[40];
    // the finishing pass may be scheduled as this grid drains (it waits for it to finish)
    asm volatile("griddepcontrol.launch_dependents;");
    const BigChunk ch = chunks[blockIdx.x];
    const BigCell C = cells[ch.big];
    const uint32_t nb = 1u << C.nbits;
    uint32_t* hist = (uint32_t*)smem;              // nb
    uint32_t* base = hist + nb;                    // nb
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    const uint32_t step = step_index(a);
    const uint32_t l_end = min(ch.l_end, min(__ldcg(&a.n_live[C.cell]), C.width));
    for (uint32_t b = tid; b < nb; b += nt) hist[b] = 0;
    __syncthreads();
    uint32_t kb[BIG_GROUPS_PER_THREAD][4];        // bucket << 16 | arrival index in the bucket
    uint32_t keys[BIG_GROUPS_PER_THREAD][4];
#pragma unroll
    for (uint32_t q = 0; q < BIG_GROUPS_PER_THREAD; ++q) {
        const uint32_t l0 = ch.l_begin + 4 * (tid + q * nt);
        U4 x = {0, 0, 0, 0};
        if (l0 < l_end) x = philox(l0 >> 2, C.cell, step, 0u, a.pk);
#pragma unroll
        for (uint32_t k = 0; k < 4; ++k) {
            keys[q][k] = u4_word(x, k);
            kb[q][k] = DEAD;
            if (l0 + k < l_end) {
                const uint32_t b = C.nbits ? keys[q][k] >> (32u - C.nbits) : 0u;
                kb[q][k] = (b << 16) | atomicAdd(&hist[b], 1u);
            }
        }
    }
    __syncthreads();
    // reserve each bucket's run with one global atomic, several in flight per thread
    for (uint32_t b0 = tid; b0 < nb; b0 += BIG_ATOMIC_ILP * nt) {
        uint32_t r[BIG_ATOMIC_ILP];
#pragma unroll
        for (uint32_t j = 0; j < BIG_ATOMIC_ILP; ++j) {
            const uint32_t b = b0 + j * nt;
            const uint32_t h = b < nb ? hist[b] : 0u;
            r[j] = h ? atomicAdd(&bk.cursor[C.bucket_base + b], h) : 0u;
        }
#pragma unroll
        for (uint32_t j = 0; j < BIG_ATOMIC_ILP; ++j)
            if (b0 + j * nt < nb) base[b0 + j * nt] = r[j];
    }
    __syncthreads();
#pragma unroll
    for (uint32_t q = 0; q < BIG_GROUPS_PER_THREAD; ++q) {
        const uint32_t l0 = ch.l_begin + 4 * (tid + q * nt);
#pragma unroll
        for (uint32_t k = 0; k < 4; ++k) {
            const uint32_t bo = kb[q][k];
            if (bo == DEAD) continue;
            const uint32_t b = bo >> 16;
            const uint32_t pos = base[b] + (bo & 0xffffu);
            if (pos < bk.cap)
                rec[(uint64_t)(C.bucket_base + b) * bk.cap + pos] = (((uint64_t)keys[q][k]) << 32) | (uint64_t)(l0 + k);
        }
    }
    // the cell's last CTA to finish turns its bucket counts into the buckets' plan and clears
    // them (the cursor atomics above returned, so they are complete before the ticket is taken)
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = (atomicAdd(&bk.ticket[ch.big], 1u) == ch.n_of_cell - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    cell_bucket_plan(bk.cursor + C.bucket_base, bk.plan + C.bucket_base, nb, bk.cap, hist, wt, a.err);
    if (tid == 0) bk.ticket[ch.big] = 0;
}

// ---------------------------------------------------------------------------
// One-dimensional bulk copies (TMA) from global into shared memory, completed on
// an mbarrier: both addresses 16-byte aligned, the size a multiple of 16 bytes.
// Every wait is bounded: after ASYNC_WAIT_CYCLES of polling the waiter gives up
// (the caller records ERR_TIMEOUT and stops).
// ---------------------------------------------------------------------------
constexpr long long ASYNC_WAIT_CYCLES = 1ll << 31;   // ~1 s at the 2.03 GHz SM clock

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// the phase's single arrival, announcing the bytes its copies deliver
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// this thread's earlier generic-proxy accesses of shared memory before later async-proxy writes
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return done != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// ---------------------------------------------------------------------------
// Large cells, pass 2: one warp per bucket -- sort it, locate it in the cell's
// order from its plan, process its pairs.  A warp takes the buckets g, g + W,
// g + 2W, ... (W warps in the grid); while one is paired, the bulk copy of the
// next one's records is in flight into the warp's record buffer.  Warps never
// wait for each other (no block barrier after the table is staged), so the
// loads of one warp overlap the arithmetic of the others.
// ---------------------------------------------------------------------------
constexpr uint32_t FQ_CAP = 64;    // finishing pass: queued pairs per warp (< 32 left + 32 new)
struct FinQueue {                  // slots of the pair's SDs, phi integer
    uint32_t s1[FQ_CAP], s2[FQ_CAP];
    unsigned long long u[FQ_CAP];
};

struct FinishLayout {
    uint32_t cap;          // records per bucket (a multiple of 32, below 2^15)
    uint32_t nsub_max;     // sub-buckets of a full bucket (a power of two >= cap)
    uint32_t warps;        // warps (buckets in flight) per CTA
    uint32_t o_rec, o_off, o_tmp, o_srt, o_cnt, o_bar, o_q, warp_bytes;   // per-warp region layout
    uint32_t o_tab, bytes;
};

// Per warp: the bucket's records in arrival order (the bulk copies' destination), each record's
// arrival index within its sub-bucket (16 bits; later, in the same bytes, the list of sub-buckets
// holding several records), the arrival indices of those records grouped by sub-bucket, the arrival
// indices in sorted order, the sub-bucket counters (16 bits, two per word), the copies' mbarrier,
// and -- when the warp evaluates its pairs itself (queue = false) -- its queue of surviving pairs.
// Once sorted, the positions in sorted order (32 bits) take the bytes of the arrival indices and
// the grouped records, and the volume bins in sorted order those of the sorted arrival indices.
__host__ __device__ inline FinishLayout finish_layout(uint32_t cap, uint32_t max_smem, bool queue = false)
{
    FinishLayout L;
    L.cap = cap;
    L.nsub_max = 1u << ceil_log2(cap > 2 ? cap : 2);                // about one record per sub-bucket
    uint32_t o = 0;
    L.o_rec = o; o = align_up(o + 8 * cap, 16);
    L.o_off = o; o = o + 2 * cap;                                   // cap is even: off and tmp are
    L.o_tmp = o; o = align_up(o + 2 * cap, 16);                     // contiguous (the positions' 4 cap)
    L.o_srt = o; o = align_up(o + 2 * cap, 16);
    L.o_cnt = o; o = align_up(o + 2 * (L.nsub_max + 2), 16);
    L.o_bar = o; o = align_up(o + 8, 16);
    L.o_q = o;
    if (!queue) o = align_up(o + (uint32_t)sizeof(FinQueue), 16);
    L.warp_bytes = o;
    L.o_tab = 0;
    const uint32_t tab = align_up((uint32_t)sizeof(EffTab), 16);
    uint32_t w = (max_smem - tab) / L.warp_bytes;
    w = w > 8 ? 8 : (w < 1 ? 1 : w);
    L.warps = w;
    L.bytes = tab + w * L.warp_bytes;
    return L;
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, v, o);
        v = t < v ? t : v;
    }
    return v;
}


// Evaluate the top 'take' queued pairs of a finishing warp (lanes < take) and pop them;
// the queue holds global slots, all of the cell whose context is cc.
__device__ __forceinline__ void fin_drain(const StepArgs& a, const EffTab* __restrict__ tab, FinQueue& Q,
                                          uint32_t& qcnt, uint32_t take, const CellCtx& cc, uint32_t* rflag,
                                          LocalStats& ls, uint32_t lane)
{
    __syncwarp();
    if (lane < take) {
        const uint32_t q = qcnt - take + lane;
        const uint64_t g1 = Q.s1[q], g2 = Q.s2[q];
        process_pair<false>(a, tab, cc, Q.u[q], g1, g2, a.xi[g1], a.xi[g2], a.attr[g1], a.attr[g2], ls, rflag);
    }
    __syncwarp();
    qcnt -= take;
}

// The warp's record buffer and its mbarrier; 'pending' while a copy into it is in flight.  extra:
// bytes each copy announces beyond those it delivers (the failure-path self-test; 0 otherwise);
// limit: the SM cycles a wait polls before it gives up.
struct FinStage {
    uint64_t* rec;
    uint64_t* bar;
    uint32_t phase;
    bool pending;
    uint32_t extra;
    long long limit;
};

// Start the bulk copy of bucket g's records (plan P) into the record buffer (lane 0 issues it);
// nothing for an empty bucket or a cell that lost records.  k <= cap and cap even, so the size
// rounded up to 16 bytes stays inside the bucket's capacity.
__device__ __forceinline__ void fin_stage(FinStage& F, const uint4& P, uint32_t g, const uint64_t* __restrict__ rec,
                                          uint32_t cap, uint32_t lane)
{
    if (P.z == BUCKET_OVERFLOWED || P.y == 0) return;
    __syncwarp();
    if (lane == 0) {
        const uint32_t bytes = 8u * ((P.y + 1u) & ~1u);
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(F.bar, bytes + F.extra);
        bulk_copy_g2s(F.rec, rec + (uint64_t)g * cap, bytes, F.bar);
    }
    F.pending = true;
}

// Wait for the copy in flight; false (ERR_TIMEOUT recorded) if it did not land in time, after a
// second bounded wait for it.
__device__ __forceinline__ bool fin_wait(FinStage& F, uint32_t* err, uint32_t lane)
{
    if (!F.pending) return true;
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(F.bar, F.phase, F.limit));
    if (!ok) {
        if (lane == 0) atomicOr(err, ERR_TIMEOUT);
        mbar_wait_bounded(F.bar, F.phase, F.limit);
    }
    F.pending = false;
    F.phase ^= 1u;
    return ok;
}

// One bucket of a large cell under the SORT contract: order its records by (key, position), locate
// it in the cell's order, and take its pairs through the early exit.  Its records are in the
// record buffer or on their way; once the bucket is sorted, the copy of the warp's next bucket gn
// (plan Pn; has_next) starts.  QUEUE: the surviving pairs go to the step's queue (evaluated by
// wc_pairs_kernel); otherwise to the warp's queue, evaluated here 32 at a time.  False: a copy did
// not land in time.
template <bool QUEUE>
__device__ __forceinline__ bool finish_bucket(const StepArgs& a, const EffTab* __restrict__ tab,
                                              const BucketDesc* __restrict__ bucket_desc,
                                              const uint64_t* __restrict__ rec, const uint4* __restrict__ plan,
                                              const unsigned long long* __restrict__ xmax, const FinishLayout& L,
                                              unsigned char* ws, uint32_t g, const uint4& P, bool has_next,
                                              uint32_t gn, const uint4& Pn, FinStage& F, uint32_t lane,
                                              uint32_t step, LocalStats& ls, uint32_t* removed, FinQueue& Q,
                                              uint32_t& qcnt, CellCtx& qcc, uint32_t& qbig, const WcQueue& W)
{
    uint64_t* srec = F.rec;                         // records in arrival order
    uint16_t* off = (uint16_t*)(ws + L.o_off);      // arrival index in the sub-bucket, then the work list
    uint16_t* tmp = (uint16_t*)(ws + L.o_tmp);      // records of shared sub-buckets, grouped
    uint16_t* srt = (uint16_t*)(ws + L.o_srt);      // arrival indices in sorted order
    uint16_t* cnt = (uint16_t*)(ws + L.o_cnt);
    uint32_t* cw = (uint32_t*)(ws + L.o_cnt);       // the counters two per word
    uint32_t* ssl = (uint32_t*)(ws + L.o_off);      // once sorted: positions in sorted order
    uint8_t* sbin = (uint8_t*)(ws + L.o_srt);       // once sorted: volume bins in sorted order
    const uint32_t cap = L.cap;
    const uint32_t S = P.x, k = P.y, n = P.z;
    if (n == BUCKET_OVERFLOWED || k == 0) {         // records were lost (the cell stays as it is), or none
        if (has_next) fin_stage(F, Pn, gn, rec, cap, lane);
        return true;
    }
    // the bucket's cell and its context, loaded ahead of the sort
    const BucketDesc C = bucket_desc[g];
    const uint32_t big = C.big;
    const uint32_t nb = 1u << C.nbits;
    const uint32_t gl = g - C.bucket_base;          // bucket in the cell
    const uint32_t kid = (uint32_t)a.kid[C.cell];
    const double dvc = a.dv[C.cell];
    const unsigned long long xm = xmax[big];
    if (!fin_wait(F, a.err, lane)) return false;
    // counting sort on the key bits below the bucket's, about one sub-bucket per record: a record
    // alone in its sub-bucket goes straight to its place; the records of a sub-bucket holding
    // several are grouped, the sub-bucket listed once (by its first arrival), and each listed
    // sub-bucket is then ordered by one lane with an insertion sort.  A record is
    // (key << 32) | position, so the order by (key, position) is the records' integer order
    // (positions differ, so no two records are equal).
    uint32_t nbb = ceil_log2(k > 2 ? k : 2);
    if (nbb > 32u - C.nbits) nbb = 32u - C.nbits;
    const uint32_t nsub = 1u << nbb;
    const uint32_t sh = 32u - nbb;
    auto sub_of = [&](uint64_t e) { return ((uint32_t)(e >> 32) << C.nbits) >> sh; };
    for (uint32_t t = lane; 2 * t < nsub; t += 32) cw[t] = 0;
    __syncwarp();
#pragma unroll 4
    for (uint32_t i = lane; i < k; i += 32) {
        const uint32_t b = sub_of(srec[i]), hs = (b & 1u) << 4;
        off[i] = (uint16_t)(atomicAdd(&cw[b >> 1], 1u << hs) >> hs);
    }
    __syncwarp();
    warp_exclusive_scan16(cnt, nsub, lane);
    uint32_t nwork = 0;
    for (uint32_t i0 = 0; i0 < k; i0 += 32) {      // warp-uniform
        const uint32_t i = i0 + lane;
        bool lead = false;
        uint32_t b = 0;
        if (i < k) {
            b = sub_of(srec[i]);
            const uint32_t st = cnt[b], c = cnt[b + 1] - st;
            const uint32_t o = off[i];
            if (c == 1) srt[st] = (uint16_t)i;
            else tmp[st + o] = (uint16_t)i;
            lead = c > 1 && o == 0;
        }
        // a list entry never lands on an arrival index still to be read
        const unsigned m = __ballot_sync(0xffffffffu, lead);
        if (lead) off[nwork + __popc(m & ((1u << lane) - 1u))] = (uint16_t)b;
        nwork += __popc(m);
    }
    __syncwarp();
    for (uint32_t w = lane; w < nwork; w += 32) {
        const uint32_t b = off[w];
        const uint32_t st = cnt[b], en = cnt[b + 1];
        for (uint32_t i = st; i < en; ++i) {
            const uint32_t p = tmp[i];
            const uint64_t ep = srec[p];
            uint32_t j = i;
            for (; j > st; --j) {
                const uint32_t q = srt[j - 1];
                if (srec[q] < ep) break;
                srt[j] = (uint16_t)q;
            }
            srt[j] = (uint16_t)p;
        }
    }
    __syncwarp();
    // positions in sorted order, and a gather of their volume bins (one byte each from the bin
    // array, else the volume's high word) put in flight for the pairs below
    const uint8_t* __restrict__ vbin = a.vbin;
    const uint32_t* attr_hi = reinterpret_cast<const uint32_t*>(a.attr) + 1;
    constexpr uint32_t FB = 8;                      // bins per lane in flight (the rest one by one)
    uint32_t bins[FB];
#pragma unroll
    for (uint32_t j = 0; j < FB; ++j) {
        const uint32_t r = lane + 32 * j;
        bins[j] = 0;
        if (r < k) {
            const uint32_t pos = (uint32_t)srec[srt[r]];
            const uint64_t e = C.slot_begin + pos;
            bins[j] = vbin ? (uint32_t)vbin[e] : pb_bin_key(attr_hi[2 * e] >> 18);
            ssl[r] = pos;
        }
    }
    for (uint32_t r = lane + 32 * FB; r < k; r += 32) ssl[r] = (uint32_t)srec[srt[r]];
    __syncwarp();
    // the record buffer is free: the next bucket's copy overlaps this one's pairs
    if (has_next) fin_stage(F, Pn, gn, rec, cap, lane);
#pragma unroll
    for (uint32_t j = 0; j < FB; ++j)
        if (lane + 32 * j < k) sbin[lane + 32 * j] = (uint8_t)bins[j];
    for (uint32_t r = lane + 32 * FB; r < k; r += 32) {
        const uint64_t e = C.slot_begin + ssl[r];
        sbin[r] = (uint8_t)(vbin ? (uint32_t)vbin[e] : pb_bin_key(attr_hi[2 * e] >> 18));
    }
    // the partner of this bucket's last SD may be the first SD of the next non-empty bucket
    unsigned long long nxt = ~0ull;
    uint32_t nxt_bin = 0;
    if (((S + k) & 1u) && (S + k < n)) {
        uint32_t b2 = gl + 1;
        while (b2 < nb && plan[C.bucket_base + b2].y == 0) ++b2;
        if (b2 < nb) {
            const uint32_t g2 = C.bucket_base + b2;
            const uint32_t k2 = plan[g2].y;
            const uint64_t* R2 = rec + (uint64_t)g2 * cap;
            for (uint32_t i = lane; i < k2; i += 32) {
                const unsigned long long e = R2[i];
                nxt = e < nxt ? e : nxt;
            }
            nxt = warp_min_u64(nxt);
            const uint64_t e = C.slot_begin + (uint32_t)nxt;
            nxt_bin = vbin ? (uint32_t)vbin[e] : pb_bin_key(attr_hi[2 * e] >> 18);
        }
    }
    __syncwarp();
    if (n < 2) return true;
    const CellCtx cc = {C.cell, n, kid, pair_ratio_dtdv_f(n, a.dt_f, dvc), dvc};
    // pairs m whose first SD (cell position 2m) lies in this bucket: 2m in [S, S+k), 2m+1 < n;
    // each lane takes two consecutive pairs (one Philox call).  The early exit needs the two
    // volumes' bins and the cell's multiplicity bound; the pairs it does not settle are queued.
    const uint32_t m_lo = (S + 1) >> 1;
    const uint32_t m_hi = min((S + k - 1) >> 1, (n >> 1) - 1);      // inclusive
    if (m_lo > m_hi) return true;
    const float c_upx = __fmul_ru(exit_scale(cc.s_dtdv32, cc.kid, a.golovin_bf, a.precision), __ull2float_ru(xm));
    const float* __restrict__ tb = g_pbound[cc.kid];
    if (!QUEUE) {
        // the warp's queue carries over from bucket to bucket of one cell (fewer, fuller drains)
        if (qcnt > 0 && qbig != big) fin_drain(a, tab, Q, qcnt, qcnt, qcc, &removed[qbig], ls, lane);
        qcc = cc;
        qbig = big;
    }
    for (uint32_t Mb = m_lo >> 1; Mb <= (m_hi >> 1); Mb += 32) {    // warp-uniform trip count
        const uint32_t M = Mb + lane;
        uint32_t sl[2][2], kv[2][2];
        bool ok[2];
#pragma unroll
        for (uint32_t h = 0; h < 2; ++h) {
            const uint32_t m = 2 * M + h;
            ok[h] = M <= (m_hi >> 1) && m >= m_lo && m <= m_hi;
            const uint32_t r = ok[h] ? 2 * m - S : 0u;
            const bool last = r + 1 >= k;              // partner is the first SD of the next bucket
            sl[h][0] = ssl[r];
            sl[h][1] = last ? (uint32_t)nxt : ssl[r + 1];
            kv[h][0] = ok[h] ? (uint32_t)sbin[r] : 0u;
            kv[h][1] = !ok[h] ? 0u : last ? nxt_bin : (uint32_t)sbin[r + 1];
        }
        uint64_t u[2] = {0, 0};
        if (M <= (m_hi >> 1)) phi_pair_u53(a, C.cell, step, M, u[0], u[1]);
        bool need[2];
#pragma unroll
        for (uint32_t h = 0; h < 2; ++h) {
            need[h] = false;
            if (ok[h]) {
                need[h] = !(__fmul_ru(__ldg(tb + pb_index(kv[h][0], kv[h][1])), c_upx) <=
                            phi_lo23((uint32_t)(u[h] >> 21)));
                ls.pairs += need[h] ? 0u : 1u;
            }
        }
        if (QUEUE) {
            // (cell, slots, pair index m | BIG) to the step's queue, one reservation per warp, lane by lane
            const unsigned m0 = __ballot_sync(0xffffffffu, need[0]), m1 = __ballot_sync(0xffffffffu, need[1]);
            const uint32_t tot = __popc(m0) + __popc(m1);
            if (tot) {
                uint32_t qb = 0;
                if (lane == 0) qb = atomicAdd(W.count, tot);
                const unsigned lt = (1u << lane) - 1u;
                qb = __shfl_sync(0xffffffffu, qb, 0) + __popc(m0 & lt) + __popc(m1 & lt);
#pragma unroll
                for (uint32_t h = 0; h < 2; ++h)
                    if (need[h])
                        W.q[qb++] = make_uint4(C.cell, C.slot_begin + sl[h][0], C.slot_begin + sl[h][1],
                                               (2 * M + h) | WQ_BIG);
            }
        } else {
#pragma unroll
            for (uint32_t h = 0; h < 2; ++h) {
                const unsigned mk = __ballot_sync(0xffffffffu, need[h]);
                if (need[h]) {
                    const uint32_t q = qcnt + __popc(mk & ((1u << lane) - 1u));
                    Q.s1[q] = C.slot_begin + sl[h][0];
                    Q.s2[q] = C.slot_begin + sl[h][1];
                    Q.u[q] = u[h];
                }
                qcnt += __popc(mk);
                if (qcnt >= 32) fin_drain(a, tab, Q, qcnt, 32, cc, &removed[big], ls, lane);
            }
        }
    }
    return true;
}

// MINB: CTAs per SM the registers are sized for -- 2 when all buckets fit one wave of warps
// (each bucket's latency is what counts), 3 when the warps take several buckets each.  QUEUE: see
// finish_bucket; the pairs' evaluation, removals and compaction then belong to wc_pairs_kernel and
// wc_compact_kernel, else to this kernel (its last CTA compacts the cells that lost SDs).
template <int MINB, bool QUEUE>
__global__ void __launch_bounds__(256, MINB) big_finish_kernel(StepArgs a, const BigCell* __restrict__ cells,
                                                         const BucketDesc* __restrict__ bucket_desc,
                                                         const uint64_t* __restrict__ rec,
                                                         const uint4* __restrict__ plan, uint32_t n_buckets,
                                                         const unsigned long long* __restrict__ xmax,
                                                         FinishLayout L, BigBook bb, WcQueue W)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long red[8];
    __shared__ uint32_t wt[40];
    EffTab* tab = (EffTab*)(smem + L.o_tab);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* ws = smem + align_up((uint32_t)sizeof(EffTab), 16) + warp * L.warp_bytes;
    const uint32_t step = step_index(a);
    LocalStats ls = {0, 0, 0, 0, 0ull};
    FinStage F{(uint64_t*)(ws + L.o_rec), (uint64_t*)(ws + L.o_bar), 0u, false, a.stage_extra,
               a.wait_log2 ? (1ll << a.wait_log2) : ASYNC_WAIT_CYCLES};
    if (lane == 0) mbar_init(F.bar);
    if (!QUEUE) load_eff_tab(tab);
    if (tid < 5) red[tid] = 0;
    __syncthreads();
    // launched as a dependent of the scatter pass: its records and plan are complete from here;
    // the pair kernel that follows may be scheduled as this grid drains
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    FinQueue& Q = *(FinQueue*)(ws + L.o_q);         // used only without QUEUE
    uint32_t qcnt = 0, qbig = 0;                   // warp-uniform
    CellCtx qcc{};
    const uint32_t stride = gridDim.x * L.warps;
    uint32_t g = blockIdx.x * L.warps + warp;
    if (g < n_buckets) {
        uint4 P = plan[g];
        fin_stage(F, P, g, rec, L.cap, lane);
        for (; g < n_buckets; g += stride) {
            const uint32_t gn = g + stride;
            const bool has_next = gn < n_buckets;
            const uint4 Pn = has_next ? plan[gn] : P;
            if (!finish_bucket<QUEUE>(a, tab, bucket_desc, rec, plan, xmax, L, ws, g, P, has_next, gn, Pn, F, lane,
                                      step, ls, bb.removed, Q, qcnt, qcc, qbig, W))
                break;
            P = Pn;
        }
        fin_wait(F, a.err, lane);                   // nothing in flight after the run (a no-op unless it broke off)
    }
    if (!QUEUE && qcnt > 0) fin_drain(a, tab, Q, qcnt, qcnt, qcc, &bb.removed[qbig], ls, lane);
    if (a.stats) {
        __syncthreads();
        flush_stats(a, ls, red);
    }
    if (!QUEUE) big_end_of_step(a, cells, bb, wt, ls.removed != 0);
}

// ---------------------------------------------------------------------------
// small utility kernels
// ---------------------------------------------------------------------------
// Per large cell: the largest multiplicity in its slots.  Coalescence never
// raises a multiplicity, so the value bounds every later step until the state
// is replaced.  One CTA per chunk of a large cell; xmax (zeroed before) takes
// the maximum over the chunks.  With vbin, also (re)writes the volume bin of
// every slot of the large cells.
__global__ void big_xmax_kernel(const uint64_t* __restrict__ xi, const double* __restrict__ vol,
                                uint8_t* __restrict__ vbin, const BigCell* __restrict__ cells,
                                const BigChunk* __restrict__ chunks, unsigned long long* xmax)
{
    __shared__ unsigned long long s_max[32];
    const BigChunk K = chunks[blockIdx.x];
    const BigCell C = cells[K.big];
    unsigned long long m = 0;
    for (uint32_t i = K.l_begin + threadIdx.x; i < K.l_end; i += blockDim.x) {
        m = max(m, (unsigned long long)xi[C.slot_begin + i]);
        if (vbin) vbin[C.slot_begin + i] = (uint8_t)vbin_of(vol[C.slot_begin + i]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (uint32_t w = 1; w < (blockDim.x + 31) / 32; ++w) m = max(m, s_max[w]);
        if (m) atomicMax(&xmax[K.big], m);
    }
}

// ---------------------------------------------------------------------------
// Displacement (sdm_rebucket): every live SD moves to the cell its new index names;
// within a cell the SDs keep their old slot order.  A stable sort of the slots by
// new cell -- least-significant-digit radix passes of 8 bits over the cell index,
// each a per-tile digit count, a scan over (digit, tile) and a stable scatter --
// then a gather into the cells' slot ranges.  Dead slots sort last (key n_cell).
// ---------------------------------------------------------------------------
constexpr uint32_t RB_TILE = 2048;            // slots per block of a radix pass
constexpr uint32_t RB_THREADS = 256;
constexpr uint32_t RB_WARPS = RB_THREADS / 32;
constexpr uint32_t RB_PER_WARP = RB_TILE / RB_WARPS;
constexpr uint32_t ERR_CAPACITY = 8u;         // a cell would receive more SDs than its width

__global__ void rb_keys_kernel(const uint64_t* __restrict__ xi, const uint32_t* __restrict__ cell_id, uint64_t n,
                               uint32_t n_cell, uint32_t* __restrict__ key, uint32_t* __restrict__ val,
                               uint32_t* __restrict__ count, uint32_t* err)
{
    uint32_t bad = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t k = n_cell;
        if (xi[i] != 0) {
            const uint32_t c = cell_id[i];
            if (c < n_cell) {
                k = c;
                atomicAdd(&count[c], 1u);
            } else {
                bad = 1;
            }
        }
        key[i] = k;
        val[i] = (uint32_t)i;
    }
    if (bad) atomicOr(err, 1u);
}

__global__ void rb_capacity_kernel(const uint32_t* __restrict__ count, const uint32_t* __restrict__ cs,
                                   uint32_t n_cell, uint32_t* err)
{
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cell; c += gridDim.x * blockDim.x)
        if (count[c] > cs[c + 1] - cs[c]) atomicOr(err, ERR_CAPACITY);
}

__global__ void __launch_bounds__(RB_THREADS) rb_hist_kernel(const uint32_t* __restrict__ key, uint64_t n,
                                                             uint32_t shift, uint32_t n_tiles,
                                                             uint32_t* __restrict__ hist)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t t0 = (uint64_t)blockIdx.x * RB_TILE;
    for (uint32_t k = threadIdx.x; k < RB_TILE; k += RB_THREADS)
        if (t0 + k < n) atomicAdd(&h[(key[t0 + k] >> shift) & 255u], 1u);
    __syncthreads();
    hist[(uint64_t)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of each digit's row of tile counts (one block per digit); tot[d] = row sum
__global__ void __launch_bounds__(RB_THREADS) rb_scan_rows_kernel(uint32_t* __restrict__ hist, uint32_t n_tiles,
                                                                  uint32_t* __restrict__ tot)
{
    __shared__ uint32_t wt[40];
    uint32_t* row = hist + (uint64_t)blockIdx.x * n_tiles;
    block_exclusive_scan(row, n_tiles, wt, false);
    if (threadIdx.x == 0) tot[blockIdx.x] = wt[32];
}

// base[d] = sum of the rows of the digits below d (one block of 256 threads)
__global__ void rb_scan_digits_kernel(const uint32_t* __restrict__ tot, uint32_t* __restrict__ base)
{
    __shared__ uint32_t s[257];
    s[threadIdx.x] = tot[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int d = 0; d < 256; ++d) {
            const uint32_t v = s[d];
            s[d] = run;
            run += v;
        }
    }
    __syncthreads();
    base[threadIdx.x] = s[threadIdx.x];
}

__global__ void __launch_bounds__(RB_THREADS) rb_scatter_kernel(const uint32_t* __restrict__ key_in,
                                                                const uint32_t* __restrict__ val_in, uint64_t n,
                                                                uint32_t shift, uint32_t n_tiles,
                                                                const uint32_t* __restrict__ hist,
                                                                const uint32_t* __restrict__ base,
                                                                uint32_t* __restrict__ key_out,
                                                                uint32_t* __restrict__ val_out)
{
    __shared__ uint32_t wc[RB_WARPS][256];       // per warp and digit: count, then offset in the tile
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    for (uint32_t k = threadIdx.x; k < RB_WARPS * 256; k += RB_THREADS) (&wc[0][0])[k] = 0;
    __syncthreads();
    const uint64_t w0 = (uint64_t)blockIdx.x * RB_TILE + (uint64_t)warp * RB_PER_WARP;
    const unsigned lt = (1u << lane) - 1u;
    for (uint32_t off = 0; off < RB_PER_WARP; off += 32) {              // the warp's digit counts
        const uint64_t i = w0 + off + lane;
        const uint32_t d = i < n ? (key_in[i] >> shift) & 255u : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (d < 256u && (peers & lt) == 0) wc[warp][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {                                                                    // warps in slot order
        uint32_t run = 0;
        for (uint32_t w = 0; w < RB_WARPS; ++w) {
            const uint32_t c = wc[w][threadIdx.x];
            wc[w][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
    for (uint32_t off = 0; off < RB_PER_WARP; off += 32) {              // stable places
        const uint64_t i = w0 + off + lane;
        const bool in = i < n;
        const uint32_t kk = in ? key_in[i] : 0u;
        const uint32_t d = in ? (kk >> shift) & 255u : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (in) {
            const uint32_t pos = base[d] + hist[(uint64_t)d * n_tiles + blockIdx.x] + wc[warp][d] + __popc(peers & lt);
            key_out[pos] = kk;
            val_out[pos] = val_in[i];
        }
        __syncwarp();
        if (in && (peers & lt) == 0) wc[warp][d] += __popc(peers);
        __syncwarp();
    }
}

// first[c] = exclusive prefix of count (one block); first[n_cell] = the live total
__global__ void rb_first_kernel(const uint32_t* __restrict__ count, uint32_t n_cell, uint32_t* __restrict__ first)
{
    __shared__ uint32_t wt[40];
    for (uint32_t c = threadIdx.x; c < n_cell; c += blockDim.x) first[c] = count[c];
    __syncthreads();
    block_exclusive_scan(first, n_cell, wt);
}

// sorted position p -> slot cs[c] + (p - first[c]) of the new cell c = key[p]; new arrays
// pre-zeroed (dead slots)
__global__ void rb_gather_kernel(const uint32_t* __restrict__ key, const uint32_t* __restrict__ val, uint64_t n,
                                 uint32_t n_cell,
                                 const uint32_t* __restrict__ first, const uint32_t* __restrict__ cs,
                                 const uint64_t* __restrict__ xi, const double* __restrict__ attr, uint64_t stride,
                                 uint32_t n_attr, uint64_t* __restrict__ xi_new, double* __restrict__ attr_new)
{
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < n; p += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = key[p], src = val[p];
        if (c >= n_cell) continue;                           // dead slots sort last
        const uint64_t dst = cs[c] + (p - first[c]);
        xi_new[dst] = xi[src];
        for (uint32_t r = 0; r < n_attr; ++r) attr_new[(uint64_t)r * stride + dst] = attr[(uint64_t)r * stride + src];
    }
}

__global__ void advance_step_kernel(uint32_t* d_step, uint32_t by)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *d_step += by;
}

__global__ void totals_kernel(const uint64_t* __restrict__ xi, const double* __restrict__ v, uint64_t n,
                              unsigned long long* out_n, double* out_mass, unsigned long long* out_live)
{
    unsigned long long sn = 0, sl = 0;
    double sm = 0.0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t x = xi[i];
        if (x) { sn += x; sl += 1; sm += (double)x * v[i]; }
    }
    sn = warp_sum(sn); sl = warp_sum(sl); sm = warp_sum(sm);
    if ((threadIdx.x & 31) == 0) {
        if (sn) atomicAdd(out_n, sn);
        if (sl) atomicAdd(out_live, sl);
        atomicAdd(out_mass, sm);
    }
}

// Mass per bin, exactly: bin b holds the live SDs with ve[b] <= v < ve[b+1].  Each term xi v is
// rounded once (the definition's terms) and is an integer multiple of 2^lsb (lsb: the unit of the
// last place of the smallest edge volume's binade); its 53-bit significand, shifted into place, is
// added as up to three 32-bit digits to 64-bit words (W per bin, word k weighing 2^(lsb + 32 k)).
// The additions are integer, so the sums do not depend on their order: per block in shared memory,
// then into acc[n_bins * W] in global memory (zeroed before); the host carries and rounds once.
// No word overflows: each holds digits below 2^32 of at most 2^32 terms.
__global__ void spectrum_exact_kernel(const uint64_t* __restrict__ xi, const double* __restrict__ v, uint64_t s0,
                                      uint64_t s1, const double* __restrict__ ve, uint32_t n_bins, int lsb,
                                      uint32_t W, unsigned long long* __restrict__ acc)
{
    extern __shared__ unsigned long long sacc[];   // [n_bins * W]
    for (uint32_t k = threadIdx.x; k < n_bins * W; k += blockDim.x) sacc[k] = 0ull;
    __syncthreads();
    for (uint64_t i = s0 + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < s1;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t x = xi[i];
        if (!x) continue;
        const double vi = v[i];
        if (!(ve[0] <= vi && vi < ve[n_bins])) continue;
        uint32_t lo = 0, hi = n_bins;          // ve[lo] <= vi < ve[hi]
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (ve[mid] <= vi) lo = mid; else hi = mid;
        }
        const double t = __dmul_rn(__ull2double_rn(x), vi);
        const uint64_t bits = (uint64_t)__double_as_longlong(t);
        const uint64_t m = (bits & ((1ull << 52) - 1ull)) | (1ull << 52);   // t >= ve[0]: a normal number
        const uint32_t o = (uint32_t)((int)((bits >> 52) & 0x7ff) - 1075 - lsb);   // t = m 2^(lsb + o)
        const uint32_t w0 = o >> 5, sh = o & 31u;
        const uint64_t lo64 = m << sh, hi64 = sh ? (m >> (64u - sh)) : 0ull;
        unsigned long long* w = sacc + lo * W + w0;
        atomicAdd(w, lo64 & 0xffffffffull);
        if (lo64 >> 32) atomicAdd(w + 1, lo64 >> 32);
        if (hi64) atomicAdd(w + 2, hi64);
    }
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < n_bins * W; k += blockDim.x)
        if (sacc[k]) atomicAdd(&acc[k], sacc[k]);
}

__global__ void eval_pairs_kernel(uint32_t kid, const double* v1, const double* v2, const uint64_t* xi1,
                                  const uint64_t* xi2, uint64_t n, uint32_t n_cell_sd, double dv, double dt,
                                  double golovin_b, double efield, double* p64, float* p32, float* err32,
                                  double* plite, double* errlite, float* pup)
{
    __shared__ EffTab tab;
    load_eff_tab(&tab);
    __syncthreads();
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t xmax = xi1[i] > xi2[i] ? xi1[i] : xi2[i];
        const double K = kernel_d(kid, v1[i], v2[i], golovin_b, efield);
        p64[i] = pair_prob_d(K, xmax, n_cell_sd, dt, dv);
        const float scale32 = u64_to_f_trunc(xmax) * pair_ratio_dtdv_f(n_cell_sd, (float)dt, dv);
        const P32 pe = pair_prob_f(&tab, kid, v1[i], v2[i], scale32, (float)golovin_b, (float)efield);
        p32[i] = pe.p;
        err32[i] = pe.err;
        if (pup) {
            const float cup = exit_scale(pair_ratio_dtdv_f(n_cell_sd, (float)dt, dv), kid, (float)golovin_b, PREC_FP64);
            pup[i] = __fmul_ru(__fmul_ru(__ldg(&g_pbound[kid][pb_index(vbin_of(v1[i]), vbin_of(v2[i]))]), cup),
                               xi_pow2_above(xi1[i], xi2[i]));
        }
        if (plite) {
            double pl = 0.0, el = -1.0;
            if (kid == 1) pair_prob_lite(v1[i], v2[i], xmax, n_cell_sd, dt, dv, pl, el);
            plite[i] = pl;
            errlite[i] = el;
        }
    }
}

__global__ void count_live_kernel(const uint64_t* __restrict__ xi, uint64_t n, unsigned long long* out)
{
    unsigned long long c = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        c += xi[i] != 0;
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

}  // namespace sdm
