// sdm_capi.cu -- host side of the C ABI declared in include/sdm.h.
//
// Owns the device state (structure-of-arrays slots grouped by cell), plans the
// device schedule (which cells are packed into shared-memory tiles and which
// go through the two-pass large-cell path), validates inputs and launches the
// kernels of sdm_kernels.cuh on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "sdm.h"
#include "sdm_kernels.cuh"

using namespace sdm;

namespace {

constexpr uint64_t XI_LIMIT = 1ull << 53;
constexpr double RHO_WATER = 1000.0;
constexpr double FOUR_PI_OVER_THREE = 4.18879020478639053;
constexpr uint32_t ERR_INVALID = 1u << 8;
constexpr uint32_t ERR_RANGE = 1u << 9;
constexpr uint32_t FINISH_SMEM = 72 * 1024;    // dynamic shared memory of a finishing CTA, three per SM
constexpr uint32_t FINISH_SMEM_WAVE = 110 * 1024;   // the same, two per SM (all buckets in one wave)
constexpr uint32_t FINISH_SMEM_MAX = 200 * 1024;   // a single-warp CTA for very wide buckets
constexpr uint32_t SCATTER_SMEM_MAX = 2 * sizeof(uint32_t) * (1u << BIG_MAX_BUCKET_BITS);
constexpr uint32_t TILE_SMEM_MAX = 227 * 1024;
constexpr uint32_t SPECTRUM_SMEM_MAX = 96 * 1024;   // the exact per-bin sums of one block

// records a bucket holds: its mean count plus ten standard deviations of the count (a
// binomial of mean m, standard deviation below sqrt(m)) plus 32; an overflow is reported
// as SDM_ECAPACITY (for m = 256: probability below 1e-20 per bucket and step)
uint32_t bucket_capacity(uint32_t mean)
{
    const uint32_t c = mean + (uint32_t)std::ceil(10.0 * std::sqrt((double)mean)) + 32;
    return (c + 31) & ~31u;
}

struct DevAlloc {
    void* p;
    size_t bytes;
};

}  // namespace

struct sdm_surrogate {
    int device = 0;
    cudaStream_t stream = nullptr;
    float* buf = nullptr;                    // w32, wbf, grad, m, v (SURR_NPS floats apart), loss
    uint8_t* mask = nullptr;                 // [SURR_TILES^2]
    float* tile_err = nullptr;               // [SURR_TILES^2]
    sdm::SurrogateDev* d_dev = nullptr;      // device copy of dev
    sdm::SurrTrainArgs args{};
    sdm::SurrogateDev dev{};
    double r_min = 0, r_max = 0;
    uint32_t steps_done = 0;
};

struct sdm_state {
    int device = 0;
    cudaStream_t stream = nullptr;
    uint64_t cap = 0;
    uint32_t n_cell = 0, n_attr = 0;
    uint64_t n_sd = 0;
    bool initialised = false;

    // memory: either owned cudaMalloc blocks or a caller workspace
    char* ws = nullptr;
    size_t ws_bytes = 0, ws_fixed = 0, ws_used = 0;
    std::vector<DevAlloc> owned_fixed, owned_layout;

    // state arrays
    uint64_t* d_xi = nullptr;
    double* d_attr = nullptr;
    uint8_t* d_vbin = nullptr;               // [cap] early-exit bin of each slot's volume
    unsigned long long* d_cell_xmax = nullptr;   // [n_cell] multiplicity bound of the cells stepped by one warp
    uint32_t* d_cell_start = nullptr;
    double* d_dv = nullptr;
    uint8_t* d_kid = nullptr;
    uint32_t* d_err = nullptr;
    unsigned long long* d_stats = nullptr;   // [5]
    unsigned long long* d_acc = nullptr;     // [4] totals scratch
    uint32_t* d_work = nullptr;              // [2] persistent tile counter
    uint32_t* d_n_live = nullptr;            // [n_cell] live SDs per cell (a prefix of its slots)

    // schedule / layout
    sdm_schedule sched{};
    TileDesc* d_tiles = nullptr;
    uint32_t n_tiles = 0, max_cells_per_tile = 0;
    uint32_t* d_wcells = nullptr;            // cells of at most WC_MAX slots, one warp each
    WcQueue wq{};                            // their queue of pairs past the early exit
    uint32_t* d_wq_ticket = nullptr;         // the compaction kernel's ticket
    uint32_t wq_grid = 0;                    // grid of the queue's pair and compaction kernels
    char* rb_buf = nullptr;                  // scratch of sdm_rebucket, kept between calls
    size_t rb_bytes = 0;
    uint32_t n_wcells = 0, wc_grid = 0, wc_grid_sort = 0;
    TileLayout tile_L{};
    BigCell* d_big = nullptr;
    uint32_t n_big = 0;
    BigChunk* d_chunks = nullptr;
    uint32_t n_chunks = 0;
    BucketDesc* d_bucket_desc = nullptr;      // [n_buckets] the cell of each SORT bucket
    uint32_t n_buckets = 0, bucket_cap = 0, max_nb = 0;
    uint32_t dbg_stage_extra = 0, dbg_wait_log2 = 0;   // sdm_debug_stage_shortfall
    uint32_t* d_cursor = nullptr;            // [n_buckets] appends per bucket (zero between steps)
    uint4* d_plan = nullptr;                 // [n_buckets] each bucket's start, records and cell total this step
    uint32_t* d_ticket = nullptr;            // [n_big] scatter CTAs of each large cell that finished
    uint64_t* d_scratch = nullptr;
    uint32_t* d_big_removed = nullptr;       // [n_big] removal flags, then the 64-bit end-of-step ticket
    uint32_t n_quads = 0, prp_grid = 0;      // PRP contract: quads of all large cells, grid size
    uint32_t prp_threads = PRP_THREADS;      // and CTA size
    bool prp_gq = false;                     // the PRP kernel's surviving pairs go to the step's queue
    uint32_t* d_cta_first = nullptr;         // [prp_grid] first large cell of each CTA (many large cells)
    unsigned long long* d_big_xmax = nullptr;   // [n_big] largest multiplicity of the cell
    // a PRP step may have left large cells flagged for Step 0 since the last compaction;
    // always assumed once a PRP step was captured into a graph (its replays are not seen here)
    bool big_deferred = false, big_deferred_always = false;
    BigLaunch prp_launch{};
    FinishLayout fin_L{};
    uint32_t fin_grid = 0, n_buckets_planned = 0, fin_minb = 3;

    // host copies of the layout
    std::vector<uint32_t> h_cell_start;
    std::vector<double> h_dv;
    std::vector<uint8_t> h_kid;
    int n_sm = 148;

    // surrogate used by SDM_PREC_SURROGATE steps (device copy of its description)
    const SurrogateDev* d_surr = nullptr;

    // optional per-kernel event timing
    bool profiling = false;
    struct Rec { int kind; cudaEvent_t e0, e1; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> ev_pool;
    uint32_t prof_launches[SDM_N_KERNEL_KINDS] = {0, 0, 0, 0};
    double prof_ms[SDM_N_KERNEL_KINDS] = {0, 0, 0, 0};
};

namespace {

sdm_status cuda_status(cudaError_t e)
{
    return e == cudaSuccess ? SDM_OK : (e == cudaErrorMemoryAllocation ? SDM_ENOMEM : SDM_ECUDA);
}

#define SDM_CUDA(call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_status(e_);   \
    } while (0)

#define SDM_TRY(call)                                    \
    do {                                                 \
        sdm_status s_ = (call);                          \
        if (s_ != SDM_OK) return s_;                     \
    } while (0)

// Each kernel's opt-in shared memory limit is set to the largest any layout uses (the
// setting is per function and process-wide; a launch uses what its own layout needs), so
// states with different layouts and the allocation-free step never undercut each other.
template <typename K>
sdm_status set_dyn_smem_limit(K* kernel, uint32_t want)
{
    int dev = 0, optin = 0;
    SDM_CUDA(cudaGetDevice(&dev));
    SDM_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa{};
    SDM_CUDA(cudaFuncGetAttributes(&fa, kernel));
    const int lim = std::min<int>((int)want, optin - (int)fa.sharedSizeBytes);   // static + dynamic <= opt-in
    SDM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    return SDM_OK;
}

sdm_status set_smem_limits()
{
    SDM_TRY(set_dyn_smem_limit(big_finish_kernel<2, true>, FINISH_SMEM_MAX));
    SDM_TRY(set_dyn_smem_limit(big_finish_kernel<3, true>, FINISH_SMEM_MAX));
    SDM_TRY(set_dyn_smem_limit(big_finish_kernel<2, false>, FINISH_SMEM_MAX));
    SDM_TRY(set_dyn_smem_limit(big_scatter_kernel, SCATTER_SMEM_MAX));
    SDM_TRY(set_dyn_smem_limit(tile_step_kernel<false, 256>, TILE_SMEM_MAX));
    SDM_TRY(set_dyn_smem_limit(tile_step_kernel<true, 256>, TILE_SMEM_MAX));
    SDM_TRY(set_dyn_smem_limit(tile_step_kernel<false, 512>, TILE_SMEM_MAX));
    SDM_TRY(set_dyn_smem_limit(tile_step_kernel<true, 512>, TILE_SMEM_MAX));
    return SDM_OK;
}

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

// allocate device memory: from the workspace (bump) or with cudaMalloc
sdm_status dev_alloc(sdm_state* st, void** out, size_t bytes, bool layout)
{
    bytes = round256(bytes + 256);   // padding: bulk prefetches may round the end up to 16 bytes
    if (st->ws) {
        if (st->ws_used + bytes > st->ws_bytes) return SDM_ENOMEM;
        *out = st->ws + st->ws_used;
        st->ws_used += bytes;
        return SDM_OK;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SDM_ENOMEM;
    }
    (layout ? st->owned_layout : st->owned_fixed).push_back({p, bytes});
    *out = p;
    return SDM_OK;
}

void free_layout(sdm_state* st)
{
    for (auto& a : st->owned_layout) cudaFree(a.p);
    st->owned_layout.clear();
    if (st->ws) st->ws_used = st->ws_fixed;
    st->d_tiles = nullptr; st->d_big = nullptr; st->d_chunks = nullptr; st->d_bucket_desc = nullptr;
    st->d_cursor = nullptr; st->d_plan = nullptr; st->d_ticket = nullptr; st->d_scratch = nullptr;
    st->d_big_removed = nullptr; st->n_quads = 0; st->d_cta_first = nullptr; st->d_big_xmax = nullptr;
    st->n_tiles = st->n_big = st->n_chunks = st->n_buckets = 0;
    st->d_wcells = nullptr; st->n_wcells = st->wc_grid = st->wc_grid_sort = 0;
    st->wq = WcQueue{}; st->d_wq_ticket = nullptr; st->wq_grid = 0;
}

template <typename T>
sdm_status upload(sdm_state* st, T** d, const std::vector<T>& h)
{
    if (h.empty()) { *d = nullptr; return SDM_OK; }
    SDM_TRY(dev_alloc(st, (void**)d, h.size() * sizeof(T), true));
    SDM_CUDA(cudaMemcpyAsync(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st->stream));
    return SDM_OK;
}

uint32_t ceil_log2_h(uint64_t w)
{
    uint32_t b = 0;
    while ((1ull << b) < w) ++b;
    return b;
}

bool is_pow2(uint32_t x) { return x && !(x & (x - 1)); }

sdm_status check_schedule(const sdm_schedule& s)
{
    if (!is_pow2(s.tile_slots) || s.tile_slots < 256 || s.tile_slots > 4096) return SDM_EINVAL;
    if (s.tile_threads < 64 || s.tile_threads > 512 || s.tile_threads % 32) return SDM_EINVAL;
    if (!is_pow2(s.bucket_target) || s.bucket_target < 64 || s.bucket_target > 2048) return SDM_EINVAL;
    if (s.persistent > 32) return SDM_EINVAL;
    return SDM_OK;
}

// Plan tiles (runs of consecutive small cells) and the large-cell buckets.
// Early-exit bound table (see pb_bin in sdm_math.cuh), computed on the host in
// double: [0][b] the bin's upper volume edge, [1][b] pi (2 r)^2 vt(r) Emax (1 + 2^-10)
// at the bin's upper radius r, Emax the largest value the interpolated efficiency takes
// over the radii and radius ratios the bins allow; both rounded up to float.
void fill_pbound_host(float (*t)[PB_SIZE])   // t[PB_KINDS]
{
    constexpr double E_h[EFF_NR * EFF_NQ] = {SDM_EFF_VALUES(SDM_AS_DOUBLE)};
    auto v_lo = [](uint32_t b) {                 // bin 0 also holds every smaller volume
        return b == 0 ? 0.0 : std::ldexp(1.0 + (double)(b % 4) / 4.0, PB_EMIN + (int)(b / 4));
    };
    auto v_hi = [](uint32_t b) { return std::ldexp(1.0 + (double)(b % 4 + 1) / 4.0, PB_EMIN + (int)(b / 4)); };
    auto radius = [](double v, double f) { return v > 0.0 ? std::cbrt(v * THREE_OVER_FOUR_PI) * f : 0.0; };
    auto vt = [](double r) {
        return r < VT_R12 ? VT_K1 * r * r : (r < VT_R23 ? VT_K2 * r : VT_K3 * std::sqrt(r));
    };
    // the kernels' interpolated efficiency (efficiency_d): bilinear on each table cell, the radius
    // clamped to the nodes' range, q to [0, 1]
    auto eff = [&](double R, double q) {
        int i = 0;
        double t = 0.0;
        if (R >= c_eff_R_h[EFF_NR - 1]) {
            i = EFF_NR - 2;
            t = 1.0;
        } else if (R > c_eff_R_h[0]) {
            while (i < EFF_NR - 2 && c_eff_R_h[i + 1] <= R) ++i;
            t = (R - c_eff_R_h[i]) / (c_eff_R_h[i + 1] - c_eff_R_h[i]);
        }
        const double s = q * 10.0;
        int j = (int)s;
        double w = s - j;
        if (j >= EFF_NQ - 1) { j = EFF_NQ - 2; w = 1.0; }
        const double e0 = E_h[i * EFF_NQ + j] + w * (E_h[i * EFF_NQ + j + 1] - E_h[i * EFF_NQ + j]);
        const double e1 = E_h[(i + 1) * EFF_NQ + j] + w * (E_h[(i + 1) * EFF_NQ + j + 1] - E_h[(i + 1) * EFF_NQ + j]);
        return e0 + t * (e1 - e0);
    };
    auto up = [](double x) {
        float f = (float)x;
        if ((double)f < x) f = std::nextafter(f, INFINITY);
        return f;
    };
    for (uint32_t b1 = 0; b1 < PB_NB; ++b1) {
        const double R_lo = radius(v_lo(b1), 1.0 - 1e-12), R_hi = radius(v_hi(b1), 1.0 + 1e-12);
        for (uint32_t d = 0; d <= PB_ND; ++d) {
            // the smaller volume's range; distances beyond b1 cannot occur (filled as bin 0)
            const uint32_t b2 = d < PB_ND ? (d <= b1 ? b1 - d : 0u) : (b1 >= PB_ND ? b1 - PB_ND : 0u);
            const double s_lo = d < PB_ND ? v_lo(b2) : 0.0, s_hi = v_hi(b2);
            t[0][b1 * PB_ROW + d] = up(v_hi(b1) + s_hi);
            const double r_lo = radius(s_lo, 1.0 - 1e-12), r_hi = std::min(radius(s_hi, 1.0 + 1e-12), R_hi);
            const double q_lo = r_lo / R_hi, q_hi = R_lo > 0.0 ? std::min(1.0, r_hi / R_lo) : 1.0;
            // the interpolant's largest value on [R_lo, R_hi] x [q_lo, q_hi]: bilinear (or constant
            // in R) on every piece the node lines cut the rectangle into, so it is reached at a
            // corner of a piece -- a point whose radius is R_lo, R_hi or a node between them and
            // whose q is q_lo, q_hi or a node between them
            double Rs[EFF_NR + 2], qs[EFF_NQ + 2];
            int nr = 0, nq = 0;
            Rs[nr++] = R_lo;
            Rs[nr++] = R_hi;
            for (int i = 0; i < EFF_NR; ++i)
                if (c_eff_R_h[i] > R_lo && c_eff_R_h[i] < R_hi) Rs[nr++] = c_eff_R_h[i];
            qs[nq++] = q_lo;
            qs[nq++] = q_hi;
            for (int j = 1; j < EFF_NQ - 1; ++j)
                if (0.1 * j > q_lo && 0.1 * j < q_hi) qs[nq++] = 0.1 * j;
            double emax = 0.0;
            for (int a = 0; a < nr; ++a)
                for (int c = 0; c < nq; ++c) emax = std::max(emax, eff(Rs[a], qs[c]));
            const double dvt = std::max(0.0, vt(R_hi) - vt(r_lo)) + 0x1p-12 * (vt(R_hi) + vt(r_hi));
            const double sr = R_hi + r_hi;
            t[1][b1 * PB_ROW + d] = up(PI_D * sr * sr * dvt * emax * (1.0 + 0x1p-10));
            t[2][b1 * PB_ROW + d] = up(PI_D * sr * sr * dvt * (1.0 + 0x1p-10));   // E_eps <= 1
        }
    }
    for (uint32_t d = 0; d <= PB_ND; ++d)
        for (uint32_t k = 0; k < PB_KINDS; ++k) t[k][PB_NB * PB_ROW + d] = INFINITY;
}

// Upload the device tables once per device (first use).
// Identity of the current device's context (a fresh one after cudaDeviceReset, which reloads the
// library's module and so its __device__ arrays), from the driver's cuCtxGetCurrent and
// cuCtxGetId, reached through the runtime so that the library links no driver stub.
sdm_status current_context_id(unsigned long long* id)
{
    typedef int (*GetCurrent)(void**);
    typedef int (*GetId)(void*, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (GetCurrent)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (GetId)f;
    });
    SDM_CUDA(cudaFree(nullptr));                 // makes the device's primary context current
    void* ctx = nullptr;
    if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, id) != 0) return SDM_ECUDA;
    return SDM_OK;
}

// The early exit's bound table (g_pbound) and the dynamic shared-memory limits, set once per
// context of each device: a context created after cudaDeviceReset gets them again.
sdm_status ensure_device_tables()
{
    static std::mutex mu;
    static unsigned long long done_ctx[64] = {};   // context id + 1 (0: none yet)
    int dev = 0;
    SDM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return SDM_ENOTSUP;
    unsigned long long ctx = 0;
    SDM_TRY(current_context_id(&ctx));
    std::lock_guard<std::mutex> lock(mu);
    if (done_ctx[dev] == ctx + 1) return SDM_OK;
    static float t[PB_KINDS][PB_SIZE];
    fill_pbound_host(t);
    SDM_CUDA(cudaMemcpyToSymbol(g_pbound, t, sizeof t));
    SDM_TRY(set_smem_limits());
    done_ctx[dev] = ctx + 1;
    return SDM_OK;
}

// CTA size of the PRP kernel for a layout with n_big large cells
uint32_t prp_threads_for(uint32_t n_big) { return n_big >= PRP_MANY_CELLS ? PRP_THREADS_MANY : PRP_THREADS; }

// whether a layout's PRP step queues its large cells' surviving pairs for the pair kernel (many
// large cells: the finer CTAs) rather than deciding them in the PRP kernel
bool prp_gq_for(uint32_t threads) { return threads == PRP_THREADS_MANY; }

// Grid of the PRP kernel: one wave of resident CTAs, at most one CTA per warp's worth of quads.
uint32_t prp_grid_size(uint32_t n_quads, int n_sm, uint32_t threads, bool gq = false)
{
    // one wave of resident blocks of either instantiation (the launch is cooperative)
    int per_sm = 0, per_sm_s = 0;
    const bool many = threads == PRP_THREADS_MANY;
    const cudaError_t e1 =
        gq     ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                 &per_sm, big_prp_kernel<false, PRP_THREADS_MANY, false, true>, (int)threads, 0)
        : many ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, big_prp_kernel<false, PRP_THREADS_MANY>,
                                                               (int)threads, 0)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, big_prp_kernel<false>, (int)threads, 0);
    const cudaError_t e2 =
        gq     ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                 &per_sm_s, big_prp_kernel<true, PRP_THREADS_MANY, false, true>, (int)threads, 0)
        : many ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_s, big_prp_kernel<true, PRP_THREADS_MANY>,
                                                               (int)threads, 0)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_s, big_prp_kernel<true>, (int)threads, 0);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        cudaGetLastError();
        per_sm = per_sm_s = 1;
    }
    per_sm = std::min(per_sm, per_sm_s);
    const uint32_t wave = (uint32_t)std::max(per_sm, 1) * (uint32_t)std::max(n_sm, 1);
    return std::max<uint32_t>(1, std::min<uint32_t>(wave, (n_quads + 31) / 32));
}

// the early exit's data from the current state: per large cell and per cell stepped by one warp,
// the multiplicity bound; the volume bin of every slot of both
sdm_status refresh_big_bounds(sdm_state* st)
{
    if (st->n_wcells) {
        const uint32_t grid = std::max<uint32_t>(1, std::min<uint32_t>((st->n_wcells + 7) / 8, 8 * st->n_sm));
        cell_bounds_kernel<<<grid, 256, 0, st->stream>>>(st->d_xi, st->d_attr, st->d_cell_start, st->d_wcells,
                                                        st->n_wcells, st->d_cell_xmax, st->d_vbin);
        SDM_CUDA(cudaGetLastError());
    }
    if (!st->n_big) return SDM_OK;
    SDM_CUDA(cudaMemsetAsync(st->d_big_xmax, 0, sizeof(unsigned long long) * st->n_big, st->stream));
    big_xmax_kernel<<<st->n_chunks, 256, 0, st->stream>>>(st->d_xi, st->d_attr, st->d_vbin, st->d_big, st->d_chunks,
                                                          st->d_big_xmax);
    SDM_CUDA(cudaGetLastError());
    return SDM_OK;
}

// The compaction that follows a PRP step (big_compact_kernel), as a programmatic
// dependent launch so that its start overlaps the end of the step.
sdm_status launch_big_compact(const StepArgs& a, const BigCell* cells, uint32_t* removed, uint32_t n_big,
                              uint32_t* sync, int n_sm, cudaStream_t stream)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(std::max<uint32_t>(1, std::min<uint32_t>(n_big, (uint32_t)std::max(n_sm, 1))));
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    SDM_CUDA(cudaLaunchKernelEx(&cfg, big_compact_kernel, a, cells, removed, n_big, sync));
    return SDM_OK;
}

// the 64-bit ticket follows the removal flags at an 8-byte aligned word, then the PRP sync words
size_t big_ticket_word(size_t n_big) { return (n_big + 1) & ~(size_t)1; }

BigBook big_book(const sdm_state* st)
{
    uint32_t* tw = st->d_big_removed + big_ticket_word(st->n_big);
    return BigBook{(unsigned long long*)tw, st->d_big_removed, st->n_big, tw + 2};
}

// The value of sum_k words[k] 2^(lsb + 32 k) (words below 2^64), rounded once to the nearest double
// (ties to even): the digits are carried into base 2^32, the leading 64 bits taken with a sticky bit
// for the rest, and the 53-bit significand rounded from them.
double exact_words_to_double(const unsigned long long* words, uint32_t W, int lsb)
{
    std::vector<uint32_t> d(W + 2, 0u);
    unsigned __int128 carry = 0;
    for (uint32_t k = 0; k < W + 2; ++k) {
        const unsigned __int128 x = carry + (k < W ? (unsigned __int128)words[k] : 0);
        d[k] = (uint32_t)x;
        carry = x >> 32;
    }
    int top = (int)W + 1;
    while (top >= 0 && d[top] == 0) --top;
    if (top < 0) return 0.0;
    // the leading 64 bits: digits top, top-1 and the high part of top-2; everything below is sticky
    const int lz = __builtin_clz(d[top]);
    const int nbits = 32 * top + (32 - lz);                 // bit length of the integer
    unsigned __int128 acc = 0;
    for (int k = top; k >= 0 && k >= top - 2; --k) acc = (acc << 32) | d[k];
    int below = 32 * std::max(0, top - 2);                  // bits of the integer not in acc
    bool sticky = false;
    for (int k = top - 3; k >= 0; --k) sticky = sticky || d[k] != 0;
    const int acc_bits = nbits - below;                     // significant bits held in acc
    uint64_t sig;
    int exp2;                                               // value = sig 2^exp2 (before rounding)
    if (acc_bits <= 53) {
        sig = (uint64_t)acc << (53 - acc_bits);
        exp2 = lsb + below - (53 - acc_bits);
    } else {
        const int drop = acc_bits - 53;
        sig = (uint64_t)(acc >> drop);
        const unsigned __int128 rest = acc & (((unsigned __int128)1 << drop) - 1);
        const unsigned __int128 half = (unsigned __int128)1 << (drop - 1);
        const bool st = sticky || (rest & (half - 1)) != 0;
        if ((rest & half) && (st || (sig & 1u))) ++sig;     // round half to even
        exp2 = lsb + below + drop;
        if (sig >> 53) { sig >>= 1; ++exp2; }               // the rounding carried into a new bit
    }
    return std::ldexp((double)sig, exp2);
}

// Clears the device error word after the host has read it.  A grid barrier that gave up
// (ERR_TIMEOUT) left its arrival count behind, which would release the next barrier early:
// it is reset too (the step that timed out left the state unspecified; see sdm.h).
sdm_status clear_device_error(sdm_state* st, uint32_t e)
{
    SDM_CUDA(cudaMemsetAsync(st->d_err, 0, sizeof(uint32_t), st->stream));
    if ((e & ERR_TIMEOUT) && st->d_big_removed)
        SDM_CUDA(cudaMemsetAsync(big_book(st).sync + 2, 0, 2 * sizeof(uint32_t), st->stream));
    return SDM_OK;
}

// the state arrays a kernel that moves SDs needs
StepArgs state_args(const sdm_state* st)
{
    StepArgs a{};
    a.xi = st->d_xi;
    a.attr = st->d_attr;
    a.vbin = st->d_vbin;
    a.stride = st->cap;
    a.n_attr = st->n_attr;
    a.cell_start = st->d_cell_start;
    a.dv = st->d_dv;
    a.kid = st->d_kid;
    a.n_live = st->d_n_live;
    a.err = st->d_err;
    return a;
}

// Compacts the large cells a PRP step left flagged (a PRP step does it itself at its start):
// before the state is read, re-laid out, or stepped under the SORT contract.
sdm_status flush_big_compaction(sdm_state* st)
{
    if (!st->n_big || !st->d_big_removed) return SDM_OK;
    if (!st->big_deferred && !st->big_deferred_always) return SDM_OK;   // no PRP step since the last one
    const BigBook bb = big_book(st);
    big_compact_kernel<<<std::max<uint32_t>(1, std::min<uint32_t>(st->n_big, (uint32_t)std::max(st->n_sm, 1))), 256,
                         0, st->stream>>>(state_args(st), st->d_big, bb.removed, st->n_big, bb.sync);
    SDM_CUDA(cudaGetLastError());
    st->big_deferred = false;
    return SDM_OK;
}

sdm_status build_layout(sdm_state* st)
{
    free_layout(st);
    const sdm_schedule& S = st->sched;
    const std::vector<uint32_t>& cs = st->h_cell_start;
    const uint32_t max_cells = std::min<uint32_t>(128, S.tile_slots);
    std::vector<TileDesc> tiles;
    std::vector<uint32_t> wcells;
    std::vector<BigCell> bigs;
    std::vector<BigChunk> chunks;
    std::vector<BucketDesc> bucket_desc;
    uint32_t n_quads = 0;
    TileDesc cur{0, 0, 0, 0};
    uint32_t cur_slots = 0;
    auto flush = [&]() {
        if (cur.n_cells && cur_slots) {
            cur.slot_end = cur.slot_begin + cur_slots;
            tiles.push_back(cur);
        }
        cur.n_cells = 0;
        cur_slots = 0;
    };
    const uint32_t tbits = ceil_log2_h(S.bucket_target);
    uint32_t bucket_cap = 0, max_nb = 1;
    for (uint32_t c = 0; c < st->n_cell; ++c) {
        const uint32_t w = cs[c + 1] - cs[c];
        if (w > S.tile_slots) {
            flush();
            BigCell b{};
            b.cell = c;
            b.slot_begin = cs[c];
            b.width = w;
            const uint32_t lw = ceil_log2_h(w);
            uint32_t nbits = lw > tbits ? lw - tbits : 0;
            nbits = std::min<uint32_t>(nbits, BIG_MAX_BUCKET_BITS);
            b.nbits = nbits;
            b.bucket_base = (uint32_t)bucket_desc.size();
            const uint32_t nb = 1u << nbits;
            for (uint32_t k = 0; k < nb; ++k)
                bucket_desc.push_back(BucketDesc{c, b.slot_begin, b.bucket_base, nbits, (uint32_t)bigs.size(), 0, 0, 0});
            const uint32_t mean = (w + nb - 1) / nb;
            bucket_cap = std::max(bucket_cap, bucket_capacity(mean));
            max_nb = std::max(max_nb, nb);
            const uint32_t n_of_cell = (w + BIG_CHUNK - 1) / BIG_CHUNK;
            for (uint32_t l = 0; l < w; l += BIG_CHUNK)
                chunks.push_back(BigChunk{(uint32_t)bigs.size(), l, std::min(w, l + BIG_CHUNK), n_of_cell});
            b.quad_begin = n_quads;
            n_quads += (w / 2 + 1) / 2;                       // quads at full occupancy
            bigs.push_back(b);
            continue;
        }
        if (w <= WC_MAX) {                   // a warp's cell (below two slots: never a pair)
            flush();
            if (w >= 2) wcells.push_back(c);
            continue;
        }
        if (cur.n_cells && (cur_slots + w > S.tile_slots || cur.n_cells == max_cells)) flush();
        if (cur.n_cells == 0) { cur.slot_begin = cs[c]; cur.cell_begin = c; }
        cur.n_cells++;
        cur_slots += w;
    }
    flush();
    bucket_cap = (bucket_cap + 31) & ~31u;
    st->n_buckets_planned = (uint32_t)bucket_desc.size();
    if (!bigs.empty()) {
        SDM_TRY(set_smem_limits());
        // two CTAs per SM (more registers: a shorter latency per bucket) unless three CTAs per SM
        // (more warps in flight) take fewer rounds of buckets per warp
        const uint32_t nbk = st->n_buckets_planned;
        const FinishLayout f2 = finish_layout(bucket_cap, FINISH_SMEM_WAVE, true);
        const FinishLayout f3 = finish_layout(bucket_cap, FINISH_SMEM, true);
        int per2 = 0, per3 = 0;
        SDM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, big_finish_kernel<2, true>, 32 * f2.warps,
                                                               f2.bytes));
        SDM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per3, big_finish_kernel<3, true>, 32 * f3.warps,
                                                               f3.bytes));
        const uint64_t w2 = (uint64_t)std::max(per2, 1) * st->n_sm * f2.warps;
        const uint64_t w3 = (uint64_t)std::max(per3, 1) * st->n_sm * f3.warps;
        const bool three = (nbk + w3 - 1) / w3 < (nbk + w2 - 1) / w2;
        const FinishLayout fl = three ? f3 : f2;
        const int per_sm = three ? per3 : per2;
        st->fin_minb = three ? 3 : 2;
        if (fl.bytes > FINISH_SMEM_MAX) return SDM_ECAPACITY;   // a cell too large for this bucket width
        st->fin_L = fl;
        const uint32_t need = (nbk + fl.warps - 1) / fl.warps;
        st->fin_grid = std::max<uint32_t>(1, std::min<uint32_t>(need, (uint32_t)std::max(per_sm, 1) * st->n_sm));
    }
    st->tile_L = tile_layout(S.tile_slots, max_cells, S.tile_threads / 32);
    st->max_cells_per_tile = max_cells;
    if (st->tile_L.bytes > TILE_SMEM_MAX) return SDM_ECAPACITY;
    SDM_TRY(upload(st, &st->d_tiles, tiles));
    SDM_TRY(upload(st, &st->d_wcells, wcells));
    st->n_wcells = (uint32_t)wcells.size();
    if (st->n_wcells) {
        int per_sm = 0;
        const uint32_t need = (st->n_wcells + WC_WARPS - 1) / WC_WARPS;
        SDM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, warp_cells_kernel<WC_SORT_PRP>,
                                                               32 * WC_WARPS, 0));
        st->wc_grid = std::max<uint32_t>(1, std::min<uint32_t>(need, (uint32_t)std::max(per_sm, 1) * st->n_sm));
        SDM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, warp_cells_kernel<WC_MAX>,
                                                               32 * WC_WARPS, 0));
        st->wc_grid_sort = std::max<uint32_t>(1, std::min<uint32_t>(need, (uint32_t)std::max(per_sm, 1) * st->n_sm));
    }
    if (!wcells.empty() || !bigs.empty()) {
        // the queue of pairs past the early exit (the cells of one warp; the large cells under the
        // SORT contract): at most one entry per candidate pair
        uint64_t qcap = 32;
        for (uint32_t c : wcells) qcap += (cs[c + 1] - cs[c]) / 2;
        for (const BigCell& b : bigs) qcap += b.width / 2;
        SDM_TRY(dev_alloc(st, (void**)&st->wq.q, sizeof(uint4) * qcap, true));
        SDM_TRY(dev_alloc(st, (void**)&st->wq.count, sizeof(uint32_t) * 4, true));   // pairs, cells, ticket, bigs
        SDM_TRY(dev_alloc(st, (void**)&st->wq.cells, sizeof(uint32_t) * std::max<size_t>(1, wcells.size()), true));
        SDM_TRY(dev_alloc(st, (void**)&st->wq.bigcells, sizeof(uint32_t) * std::max<size_t>(1, bigs.size()), true));
        SDM_TRY(dev_alloc(st, (void**)&st->wq.flag, sizeof(uint32_t) * st->n_cell, true));
        SDM_CUDA(cudaMemsetAsync(st->wq.count, 0, sizeof(uint32_t) * 4, st->stream));
        SDM_CUDA(cudaMemsetAsync(st->wq.flag, 0, sizeof(uint32_t) * st->n_cell, st->stream));
        st->d_wq_ticket = st->wq.count + 2;
        st->wq_grid = 8 * st->n_sm;
    }
    SDM_TRY(upload(st, &st->d_big, bigs));
    SDM_TRY(upload(st, &st->d_chunks, chunks));
    SDM_TRY(upload(st, &st->d_bucket_desc, bucket_desc));
    st->n_quads = n_quads;
    if (n_quads) {
        st->prp_threads = prp_threads_for((uint32_t)bigs.size());
        st->prp_gq = prp_gq_for(st->prp_threads);
        st->prp_grid = prp_grid_size(n_quads, st->n_sm, st->prp_threads, st->prp_gq);
        std::vector<uint32_t> first(st->prp_grid);
        for (uint32_t b = 0, c = 0; b < st->prp_grid; ++b) {
            const uint32_t qa = (uint32_t)(((uint64_t)b * n_quads) / st->prp_grid);
            while (c + 1 < bigs.size() && bigs[c + 1].quad_begin <= qa) ++c;
            first[b] = c;
        }
        SDM_TRY(upload(st, &st->d_cta_first, first));
    }
    if (!bigs.empty()) {
        const size_t words = big_ticket_word(bigs.size()) + 2 + BIG_SYNC_WORDS;   // flags, ticket, PRP sync words
        SDM_TRY(dev_alloc(st, (void**)&st->d_big_removed, sizeof(uint32_t) * words, true));
        SDM_CUDA(cudaMemsetAsync(st->d_big_removed, 0, sizeof(uint32_t) * words, st->stream));
    }
    st->big_deferred = false;
    st->n_tiles = (uint32_t)tiles.size();
    st->n_big = (uint32_t)bigs.size();
    if (!bigs.empty())
        SDM_TRY(dev_alloc(st, (void**)&st->d_big_xmax, sizeof(unsigned long long) * bigs.size(), true));
    st->prp_launch = BigLaunch{st->n_big, n_quads, st->d_big, st->d_big_xmax, st->d_cta_first, {}};
    for (uint32_t b = 0; b < st->n_big && b < BIG_PARAM_CELLS; ++b) st->prp_launch.pc[b] = bigs[b];
    st->n_chunks = (uint32_t)chunks.size();
    st->n_buckets = (uint32_t)bucket_desc.size();
    st->bucket_cap = bucket_cap;
    st->max_nb = max_nb;
    if (st->n_buckets) {
        // cursors (n_buckets) and the per-cell tickets (n_big), zeroed once here; afterwards the
        // scatter pass leaves them at zero at the end of every step; the buckets' plan; the
        // records
        const size_t words = (size_t)st->n_buckets + (size_t)st->n_big;
        SDM_TRY(dev_alloc(st, (void**)&st->d_cursor, sizeof(uint32_t) * words, true));
        SDM_CUDA(cudaMemsetAsync(st->d_cursor, 0, sizeof(uint32_t) * words, st->stream));
        st->d_ticket = st->d_cursor + st->n_buckets;
        SDM_TRY(dev_alloc(st, (void**)&st->d_plan, sizeof(uint4) * (size_t)st->n_buckets, true));
        SDM_CUDA(cudaMemsetAsync(st->d_plan, 0, sizeof(uint4) * (size_t)st->n_buckets, st->stream));
        SDM_TRY(dev_alloc(st, (void**)&st->d_scratch, sizeof(uint64_t) * (size_t)st->n_buckets * bucket_cap, true));
    }
    SDM_TRY(set_smem_limits());
    SDM_CUDA(cudaStreamSynchronize(st->stream));
    return SDM_OK;
}

// host-side validation of an initial state
sdm_status validate_host(const sdm_state* st, const uint64_t* xi, const double* attr, uint64_t n)
{
    for (uint64_t i = 0; i < n; ++i) {
        if (xi[i] >= XI_LIMIT) return SDM_ERANGE;
        for (uint32_t a = 0; a < st->n_attr; ++a) {
            const double v = attr[(uint64_t)a * n + i];
            if (!std::isfinite(v)) return SDM_EINVAL;
            if (a == 0 && xi[i] != 0 && !(v > 0.0)) return SDM_EINVAL;
        }
    }
    return SDM_OK;
}

sdm_status set_cells(sdm_state* st, const std::vector<uint32_t>& cs, const double* dv, const uint8_t* kid)
{
    st->h_cell_start = cs;
    st->h_dv.assign(dv, dv + st->n_cell);
    st->h_kid.assign(st->n_cell, 0);
    if (kid) st->h_kid.assign(kid, kid + st->n_cell);
    for (uint32_t c = 0; c < st->n_cell; ++c) {
        if (!(st->h_dv[c] > 0.0) || !std::isfinite(st->h_dv[c])) return SDM_EINVAL;
        if (st->h_kid[c] > SDM_KERNEL_ELECTRIC) return SDM_EINVAL;
    }
    SDM_CUDA(cudaMemcpyAsync(st->d_cell_start, cs.data(), sizeof(uint32_t) * (st->n_cell + 1), cudaMemcpyHostToDevice,
                             st->stream));
    SDM_CUDA(cudaMemcpyAsync(st->d_dv, st->h_dv.data(), sizeof(double) * st->n_cell, cudaMemcpyHostToDevice, st->stream));
    SDM_CUDA(cudaMemcpyAsync(st->d_kid, st->h_kid.data(), st->n_cell, cudaMemcpyHostToDevice, st->stream));
    return SDM_OK;
}

// copy the slot arrays (already grouped by cell) to the device
sdm_status upload_slots(sdm_state* st, const uint64_t* xi, const double* attr, uint64_t n)
{
    SDM_CUDA(cudaMemcpyAsync(st->d_xi, xi, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, st->stream));
    for (uint32_t a = 0; a < st->n_attr; ++a)
        SDM_CUDA(cudaMemcpyAsync(st->d_attr + (uint64_t)a * st->cap, attr + (uint64_t)a * n, sizeof(double) * n,
                                 cudaMemcpyHostToDevice, st->stream));
    return SDM_OK;
}

template <typename T>
sdm_status to_host(std::vector<T>& h, const T* p, uint64_t n, int on_device, cudaStream_t s)
{
    h.resize(n);
    if (!n) return SDM_OK;
    if (on_device) {
        SDM_CUDA(cudaMemcpyAsync(h.data(), p, sizeof(T) * n, cudaMemcpyDeviceToHost, s));
        SDM_CUDA(cudaStreamSynchronize(s));
    } else {
        std::memcpy(h.data(), p, sizeof(T) * n);
    }
    return SDM_OK;
}

sdm_status init_common(sdm_state* st, const uint64_t* xi_in, const double* attr_in, const std::vector<uint32_t>& cs,
                       uint64_t n, const double* dv, const uint8_t* kid)
{
    SDM_TRY(validate_host(st, xi_in, attr_in, n));
    // stable compaction of every cell: live SDs first, in input order; removed slots zeroed
    std::vector<uint64_t> xi(n, 0);
    std::vector<double> attr((size_t)n * st->n_attr, 0.0);
    std::vector<uint32_t> n_live(st->n_cell, 0);
    for (uint32_t c = 0; c < st->n_cell; ++c) {
        uint64_t dst = cs[c];
        for (uint64_t i = cs[c]; i < cs[c + 1]; ++i) {
            if (xi_in[i] == 0) continue;
            xi[dst] = xi_in[i];
            for (uint32_t a = 0; a < st->n_attr; ++a) attr[(uint64_t)a * n + dst] = attr_in[(uint64_t)a * n + i];
            ++dst;
        }
        n_live[c] = (uint32_t)(dst - cs[c]);
    }
    SDM_TRY(set_cells(st, cs, dv, kid));
    SDM_TRY(upload_slots(st, xi.data(), attr.data(), n));
    SDM_CUDA(cudaMemcpyAsync(st->d_n_live, n_live.data(), sizeof(uint32_t) * st->n_cell, cudaMemcpyHostToDevice,
                             st->stream));
    SDM_CUDA(cudaStreamSynchronize(st->stream));
    st->n_sd = n;
    SDM_CUDA(cudaMemsetAsync(st->d_err, 0, sizeof(uint32_t), st->stream));
    SDM_TRY(build_layout(st));
    SDM_TRY(refresh_big_bounds(st));
    st->initialised = true;
    return SDM_OK;
}

// largest c with cs[c] <= i
__device__ uint32_t cell_of(const uint32_t* cs, uint32_t n_cell, uint64_t i)
{
    uint32_t lo = 0, hi = n_cell;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (cs[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void validate_kernel(const uint64_t* __restrict__ xi, const double* __restrict__ attr, uint64_t n,
                                uint64_t stride, uint32_t n_attr, const uint32_t* __restrict__ cs, uint32_t n_cell,
                                uint32_t* err)
{
    uint32_t bad = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t x = xi[i];
        if (x >= XI_LIMIT) bad |= ERR_RANGE;
        // live SDs must precede the removed slots of their cell
        if (x != 0 && i > 0 && xi[i - 1] == 0 && cs[cell_of(cs, n_cell, i)] != i) bad |= ERR_INVALID;
        for (uint32_t a = 0; a < n_attr; ++a) {
            const double v = attr[(uint64_t)a * stride + i];
            if (!isfinite(v) || (a == 0 && x != 0 && !(v > 0.0))) bad |= ERR_INVALID;
        }
    }
    if (bad) atomicOr(err, bad);
}

// state checks (sdm_check_state): slots breaking the live-prefix rule of their cell
__global__ void check_live_kernel(const uint64_t* __restrict__ xi, uint64_t n, const uint32_t* __restrict__ cs,
                                  uint32_t n_cell, const uint32_t* __restrict__ n_live, unsigned long long* bad)
{
    unsigned long long b = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = cell_of(cs, n_cell, i);
        const bool expect_live = i - cs[c] < n_live[c];
        b += (xi[i] != 0) != expect_live;
    }
    if (b) atomicAdd(bad, b);
}

// state checks: slots of the large cells whose stored volume bin is stale
__global__ void check_keys_kernel(const double* __restrict__ vol, const uint8_t* __restrict__ vbin,
                                  const BigCell* __restrict__ cells, const BigChunk* __restrict__ chunks,
                                  unsigned long long* bad)
{
    const BigChunk K = chunks[blockIdx.x];
    const BigCell C = cells[K.big];
    unsigned long long b = 0;
    for (uint32_t i = K.l_begin + threadIdx.x; i < K.l_end; i += blockDim.x)
        b += vbin[C.slot_begin + i] != (uint8_t)vbin_of(vol[C.slot_begin + i]);
    if (b) atomicAdd(bad, b);
}

// the cells stepped by one warp: slots whose stored volume bin differs from the volume's, or whose
// multiplicity exceeds the cell's bound (one warp per cell)
__global__ void check_wcell_keys_kernel(const uint64_t* __restrict__ xi, const double* __restrict__ vol,
                                        const uint8_t* __restrict__ vbin, const uint32_t* __restrict__ cs,
                                        const uint32_t* __restrict__ cells, uint32_t n_cells,
                                        const unsigned long long* __restrict__ xmax, unsigned long long* bad)
{
    const uint32_t lane = threadIdx.x & 31;
    unsigned long long b = 0;
    for (uint32_t k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n_cells; k += (gridDim.x * blockDim.x) >> 5) {
        const uint32_t c = cells[k];
        for (uint32_t i = cs[c] + lane; i < cs[c + 1]; i += 32)
            b += (vbin[i] != (uint8_t)vbin_of(vol[i])) || (xi[i] > xmax[c]);
    }
    if (b) atomicAdd(bad, b);
}

// live count of every cell: the length of the live prefix of its slots
__global__ void live_count_kernel(const uint64_t* __restrict__ xi, const uint32_t* __restrict__ cs, uint32_t n_cell,
                                  uint32_t* n_live)
{
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cell; c += gridDim.x * blockDim.x) {
        uint64_t lo = cs[c], hi = cs[c + 1];          // first removed slot in [lo, hi]
        while (lo < hi) {
            const uint64_t mid = (lo + hi) >> 1;
            if (xi[mid] != 0) lo = mid + 1; else hi = mid;
        }
        n_live[c] = (uint32_t)(lo - cs[c]);
    }
}

sdm_status err_to_status(uint32_t e)
{
    if (!e) return SDM_OK;
    if (e & ERR_RANGE) return SDM_ERANGE;
    if (e & ERR_INVALID) return SDM_EINVAL;
    if (e & (ERR_BUCKET_OVERFLOW | ERR_TILE_OVERFLOW)) return SDM_ECAPACITY;
    if (e & ERR_TIMEOUT) return SDM_ETIMEOUT;
    return SDM_ECUDA;
}

cudaEvent_t pooled_event(sdm_state* st)
{
    if (!st->ev_pool.empty()) {
        cudaEvent_t e = st->ev_pool.back();
        st->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct ProfScope {
    sdm_state* st;
    int kind;
    cudaEvent_t e0 = nullptr;
    ProfScope(sdm_state* s, int k) : st(s), kind(k)
    {
        if (st->profiling) {
            e0 = pooled_event(st);
            cudaEventRecord(e0, st->stream);
        }
    }
    ~ProfScope()
    {
        if (e0) {
            cudaEvent_t e1 = pooled_event(st);
            cudaEventRecord(e1, st->stream);
            st->recs.push_back({kind, e0, e1});
        }
    }
};

void collect_profile(sdm_state* st)
{
    if (st->recs.empty()) return;
    cudaStreamSynchronize(st->stream);
    for (auto& r : st->recs) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.e0, r.e1);
        st->prof_ms[r.kind] += ms;
        st->prof_launches[r.kind] += 1;
        st->ev_pool.push_back(r.e0);
        st->ev_pool.push_back(r.e1);
    }
    st->recs.clear();
}

sdm_status launch_steps(sdm_state* st, const sdm_step_params* p, uint32_t n_steps, bool with_stats)
{
    StepArgs a{};
    a.xi = st->d_xi;
    a.attr = st->d_attr;
    a.vbin = st->d_vbin;
    a.stride = st->cap;
    a.n_attr = st->n_attr;
    a.precision = p->precision;
    a.cell_start = st->d_cell_start;
    a.dv = st->d_dv;
    a.kid = st->d_kid;
    a.dt = p->dt;
    a.golovin_b = p->golovin_b;
    a.dt_f = (float)p->dt;
    a.golovin_bf = (float)p->golovin_b;
    a.efield = p->efield;
    a.efield_f = (float)p->efield;
    a.seed_lo = (uint32_t)(p->seed & 0xffffffffu);
    a.seed_hi = (uint32_t)(p->seed >> 32);
    a.pk = philox_keys_host(a.seed_lo, a.seed_hi);
    a.d_step = p->d_step;
    a.shuffle = p->shuffle;
    a.n_live = st->d_n_live;
    a.cell_xmax = st->d_cell_xmax;
    a.stats = with_stats ? st->d_stats : nullptr;
    a.err = st->d_err;
    a.surr = st->d_surr;
    a.stage_extra = st->dbg_stage_extra;
    a.wait_log2 = st->dbg_wait_log2;
    const sdm_schedule& S = st->sched;
    const uint32_t scatter_smem = sizeof(uint32_t) * 2 * st->max_nb;
    for (uint32_t s = 0; s < n_steps; ++s) {
        a.step = p->step + s;
        // the queued pairs, then the cells that lost SDs: launched once per step, after the kernels
        // that fill the queue, as programmatic dependents (their blocks may be scheduled while the
        // previous kernel drains; each waits for it with griddepcontrol.wait)
        const bool sort_big = st->n_big && p->shuffle == SDM_SHUFFLE_SORT;
        const bool prp_gq = st->n_big && p->shuffle == SDM_SHUFFLE_PRP && st->prp_gq;
        const bool queue_after_big = sort_big || prp_gq;
        auto launch_queue = [&]() -> sdm_status {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            at[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            cfg.stream = st->stream;
            cfg.blockDim = dim3(256);
            cfg.gridDim = dim3(st->wq_grid);
            const bool surr = p->precision == SDM_PREC_SURROGATE;
            SDM_CUDA(cudaLaunchKernelEx(&cfg, surr ? wc_pairs_kernel<true> : wc_pairs_kernel<false>, a, st->wq));
            cfg.gridDim = dim3(std::max(st->n_sm, 1));           // one block per SM: one ticket each
            SDM_CUDA(cudaLaunchKernelEx(&cfg, wc_compact_kernel, a, st->wq, st->d_wq_ticket));
            return SDM_OK;
        };
        if (st->n_wcells || st->n_tiles) {
            ProfScope ps(st, 0);
            const bool surr = p->precision == SDM_PREC_SURROGATE;
            if (st->n_wcells) {
                // shuffle and early exit per cell; the pairs it cannot settle go to the queue
                if (p->shuffle == SDM_SHUFFLE_SORT)       // lists up to 512 SDs sorted by key
                    warp_cells_kernel<WC_MAX><<<st->wc_grid_sort, 32 * WC_WARPS, 0, st->stream>>>(
                        a, st->wq, st->d_wcells, st->n_wcells);
                else                                      // above 256 SDs the keyed bijection
                    warp_cells_kernel<WC_SORT_PRP><<<st->wc_grid, 32 * WC_WARPS, 0, st->stream>>>(
                        a, st->wq, st->d_wcells, st->n_wcells);
                if (!queue_after_big) SDM_TRY(launch_queue());
            }
            if (st->n_tiles) {
                uint32_t grid = st->n_tiles;
                uint32_t* work = nullptr;
                if (S.persistent) {
                    grid = std::min<uint32_t>(st->n_tiles, S.persistent * (uint32_t)st->n_sm);
                    work = st->d_work;
                }
                auto kern = S.tile_threads <= 256
                                ? (surr ? tile_step_kernel<true, 256> : tile_step_kernel<false, 256>)
                                : (surr ? tile_step_kernel<true, 512> : tile_step_kernel<false, 512>);
                kern<<<grid, S.tile_threads, st->tile_L.bytes, st->stream>>>(a, st->d_tiles, st->n_tiles, st->tile_L,
                                                                            work);
            }
        }
        const BigBook bb = big_book(st);
        if (st->n_big && p->shuffle == SDM_SHUFFLE_PRP) {
            // cooperative: a step that finds cells flagged by the previous one compacts them first,
            // behind a grid barrier (every block resident)
            ProfScope ps(st, 3);
            if (!prp_gq) {      // cells that lose SDs stay flagged until the next launch's Step 0
                st->big_deferred = true;
                cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
                SDM_CUDA(cudaStreamIsCapturing(st->stream, &cap_status));
                if (cap_status != cudaStreamCaptureStatusNone) st->big_deferred_always = true;
            }
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(st->prp_grid);
            cfg.blockDim = dim3(st->prp_threads);
            cfg.dynamicSmemBytes = 0;
            cfg.stream = st->stream;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeCooperative;
            at[0].val.cooperative = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            const bool surr = p->precision == SDM_PREC_SURROGATE;
            if (prp_gq) {
                SDM_CUDA(cudaLaunchKernelEx(&cfg, surr ? big_prp_kernel<true, PRP_THREADS_MANY, false, true>
                                                       : big_prp_kernel<false, PRP_THREADS_MANY, false, true>,
                                            a, st->prp_launch, bb, st->wq));
                SDM_TRY(launch_queue());                 // the large cells' (and small cells') queued pairs
            } else if (st->prp_threads == PRP_THREADS_MANY) {
                SDM_CUDA(cudaLaunchKernelEx(&cfg, surr ? big_prp_kernel<true, PRP_THREADS_MANY>
                                                       : big_prp_kernel<false, PRP_THREADS_MANY>,
                                            a, st->prp_launch, bb, WcQueue{}));
            } else {
                SDM_CUDA(cudaLaunchKernelEx(&cfg, surr ? big_prp_kernel<true> : big_prp_kernel<false>, a,
                                            st->prp_launch, bb, WcQueue{}));
            }
        } else if (st->n_big) {
            SDM_TRY(flush_big_compaction(st));      // cells left flagged by a PRP step
            const BucketBook bk{st->d_cursor, st->d_plan, st->d_ticket, st->n_buckets, st->bucket_cap};
            {
                ProfScope ps(st, 1);
                big_scatter_kernel<<<st->n_chunks, BIG_SCATTER_THREADS, scatter_smem, st->stream>>>(
                    a, st->d_big, st->d_chunks, st->d_scratch, bk);
            }
            {
                ProfScope ps(st, 2);
                auto fk = st->fin_minb == 2 ? big_finish_kernel<2, true> : big_finish_kernel<3, true>;
                cudaLaunchConfig_t cfg = {};
                cudaLaunchAttribute at[1];
                at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;   // waits for the scatter
                at[0].val.programmaticStreamSerializationAllowed = 1;
                cfg.attrs = at;
                cfg.numAttrs = 1;
                cfg.stream = st->stream;
                cfg.gridDim = dim3(st->fin_grid);
                cfg.blockDim = dim3(32 * st->fin_L.warps);
                cfg.dynamicSmemBytes = st->fin_L.bytes;
                SDM_CUDA(cudaLaunchKernelEx(&cfg, fk, a, (const BigCell*)st->d_big, (const BucketDesc*)st->d_bucket_desc,
                                            (const uint64_t*)st->d_scratch, (const uint4*)st->d_plan, st->n_buckets,
                                            (const unsigned long long*)st->d_big_xmax, st->fin_L, bb, st->wq));
                SDM_TRY(launch_queue());                 // the large cells' (and small cells') queued pairs
            }
        }
        if (p->d_step) advance_step_kernel<<<1, 32, 0, st->stream>>>(p->d_step, 1u);
        SDM_CUDA(cudaGetLastError());
    }
    return SDM_OK;
}

}  // namespace

extern "C" {

const char* sdm_version(void) { return "sdm-b300 1.0 (sm_103a)"; }

const char* sdm_status_str(sdm_status s)
{
    switch (s) {
    case SDM_OK: return "SDM_OK";
    case SDM_EINVAL: return "SDM_EINVAL: invalid argument or state";
    case SDM_ENOMEM: return "SDM_ENOMEM: out of memory";
    case SDM_ECAPACITY: return "SDM_ECAPACITY: capacity exceeded";
    case SDM_ERANGE: return "SDM_ERANGE: multiplicity >= 2^53";
    case SDM_ECUDA: return "SDM_ECUDA: CUDA runtime error";
    case SDM_ETIMEOUT: return "SDM_ETIMEOUT: bounded wait expired";
    case SDM_ENOTSUP: return "SDM_ENOTSUP: not supported";
    }
    return "unknown sdm_status";
}

size_t sdm_workspace_bytes(uint64_t cap, uint32_t n_cell, uint32_t n_attr)
{
    size_t b = 0;
    b += round256(8 * cap + 256) + round256(8 * cap * n_attr + 256) + round256(cap + 256);
    b += round256(4 * ((size_t)n_cell + 1) + 256) + round256(8 * (size_t)n_cell + 256) + round256(n_cell + 256);
    b += 4 * round256(512) + round256(4 * (size_t)n_cell + 256);
    b += round256(4 * (size_t)n_cell + 260);
    b += round256(8 * (size_t)n_cell + 256);                    // multiplicity bound per cell
    // layout: tiles and big cells (<= n_cell each), chunks, buckets, cursors, scratch
    b += round256(sizeof(TileDesc) * (size_t)n_cell + 256) + round256(sizeof(BigCell) * (size_t)n_cell + 256);
    b += round256(4 * (size_t)n_cell + 256);   // cells stepped by one warp each
    // their queue (an entry per candidate pair), its counters, listed cells and flags
    b += round256(16 * (cap / 2 + 32) + 256) + round256(16 + 256) + 3 * round256(4 * (size_t)n_cell + 256);
    b += round256(sizeof(BigChunk) * (cap / BIG_CHUNK + n_cell + 1) + 256);
    const size_t max_buckets = 3 * cap / 64 + 1;
    const size_t max_cap = 2 * 2048 + 64 + 32;
    b += round256(sizeof(BucketDesc) * max_buckets + 256) + round256(16 * max_buckets + 256);   // descriptors, cursors
    b += round256(sizeof(uint4) * max_buckets + 256);                                           // plan
    b += round256(8 * max_buckets * max_cap + 256);
    return b;
}

sdm_status sdm_alloc(sdm_state** out, uint64_t cap, uint32_t n_cell, uint32_t n_attr, void* cuda_stream,
                     void* workspace, size_t ws_bytes)
{
    if (!out) return SDM_EINVAL;
    *out = nullptr;
    if (cap == 0 || cap >= (1ull << 32) || n_cell == 0 || n_attr == 0 || n_attr > 64) return SDM_EINVAL;
    sdm_state* st = new (std::nothrow) sdm_state();
    if (!st) return SDM_ENOMEM;
    st->stream = (cudaStream_t)cuda_stream;
    st->cap = cap;
    st->n_cell = n_cell;
    st->n_attr = n_attr;
    st->sched = sdm_schedule{1024, 256, 256, 0};
    if (cudaGetDevice(&st->device) != cudaSuccess) { delete st; return SDM_ECUDA; }
    cudaDeviceGetAttribute(&st->n_sm, cudaDevAttrMultiProcessorCount, st->device);
    if (workspace) {
        st->ws = (char*)(((uintptr_t)workspace + 255) & ~(uintptr_t)255);
        const size_t skew = (size_t)(st->ws - (char*)workspace);
        if (ws_bytes <= skew) { delete st; return SDM_ENOMEM; }
        st->ws_bytes = ws_bytes - skew;
    }
    sdm_status s = SDM_OK;
    if (s == SDM_OK) s = ensure_device_tables();
    if (s == SDM_OK) s = dev_alloc(st, (void**)&st->d_xi, sizeof(uint64_t) * cap, false);
    if (s == SDM_OK) s = dev_alloc(st, (void**)&st->d_attr, sizeof(double) * cap * n_attr, false);
    if (s == SDM_OK) s = dev_alloc(st, (void**)&st->d_vbin, sizeof(uint8_t) * cap, false);
    if (s == SDM_OK) s = dev_alloc(st, (void**)&st->d_cell_start, sizeof(uint32_t) * ((size_t)n_cell + 1), false);
    if (s == SDM_OK) s = dev_alloc(st, (void**)&st->d_dv, sizeof(double) * n_cell, false);
    if (s == SDM_OK) s = dev_alloc(st, (void**)&st->d_kid, n_cell, false);
    if (s == SDM_OK) s = dev_alloc(st, (void**)&st->d_err, 64, false);
    if (s == SDM_OK) s = dev_alloc(st, (void**)&st->d_stats, 64, false);
    if (s == SDM_OK) s = dev_alloc(st, (void**)&st->d_acc, 64, false);
    if (s == SDM_OK) s = dev_alloc(st, (void**)&st->d_work, 64, false);
    if (s == SDM_OK) s = dev_alloc(st, (void**)&st->d_n_live, sizeof(uint32_t) * n_cell, false);
    if (s == SDM_OK) s = dev_alloc(st, (void**)&st->d_cell_xmax, sizeof(unsigned long long) * n_cell, false);
    if (s == SDM_OK && cudaMemsetAsync(st->d_err, 0, 64, st->stream) != cudaSuccess) s = SDM_ECUDA;
    if (s == SDM_OK && cudaMemsetAsync(st->d_work, 0, 64, st->stream) != cudaSuccess) s = SDM_ECUDA;
    if (s == SDM_OK && cudaMemsetAsync(st->d_xi, 0, sizeof(uint64_t) * cap, st->stream) != cudaSuccess) s = SDM_ECUDA;
    if (s == SDM_OK && cudaStreamSynchronize(st->stream) != cudaSuccess) s = SDM_ECUDA;
    if (s != SDM_OK) { sdm_free(st); return s; }
    st->ws_fixed = st->ws_used;
    *out = st;
    return SDM_OK;
}

void sdm_free(sdm_state* st)
{
    if (!st) return;
    if (st->stream) cudaStreamSynchronize(st->stream);
    free_layout(st);
    for (auto& a : st->owned_fixed) cudaFree(a.p);
    if (st->rb_buf) cudaFree(st->rb_buf);
    collect_profile(st);
    for (auto e : st->ev_pool) cudaEventDestroy(e);
    delete st;
}

sdm_status sdm_init_state(sdm_state* st, const uint64_t* xi, const double* attr, const uint32_t* cell_id,
                          uint64_t n_sd, const double* dv, const uint8_t* kernel_id, int on_dev)
{
    if (!st || !xi || !attr || !cell_id || !dv) return SDM_EINVAL;
    if (n_sd > st->cap) return SDM_ECAPACITY;
    std::vector<uint64_t> hx;
    std::vector<double> ha, hdv;
    std::vector<uint32_t> hc;
    std::vector<uint8_t> hk;
    SDM_TRY(to_host(hx, xi, n_sd, on_dev, st->stream));
    SDM_TRY(to_host(ha, attr, n_sd * st->n_attr, on_dev, st->stream));
    SDM_TRY(to_host(hc, cell_id, n_sd, on_dev, st->stream));
    SDM_TRY(to_host(hdv, dv, st->n_cell, on_dev, st->stream));
    if (kernel_id) SDM_TRY(to_host(hk, kernel_id, st->n_cell, on_dev, st->stream));
    // stable counting sort by cell: slot order inside a cell is the input order
    std::vector<uint32_t> cs(st->n_cell + 1, 0);
    for (uint64_t i = 0; i < n_sd; ++i) {
        if (hc[i] >= st->n_cell) return SDM_EINVAL;
        cs[hc[i] + 1]++;
    }
    for (uint32_t c = 0; c < st->n_cell; ++c) cs[c + 1] += cs[c];
    std::vector<uint32_t> pos(cs.begin(), cs.end() - 1);
    std::vector<uint64_t> sx(n_sd);
    std::vector<double> sa(n_sd * st->n_attr);
    for (uint64_t i = 0; i < n_sd; ++i) {
        const uint32_t d = pos[hc[i]]++;
        sx[d] = hx[i];
        for (uint32_t a = 0; a < st->n_attr; ++a) sa[(uint64_t)a * n_sd + d] = ha[(uint64_t)a * n_sd + i];
    }
    return init_common(st, sx.data(), sa.data(), cs, n_sd, hdv.data(), kernel_id ? hk.data() : nullptr);
}

sdm_status sdm_init_state_segmented(sdm_state* st, const uint64_t* xi, const double* attr, const uint32_t* cell_start,
                                    uint64_t n_sd, const double* dv, const uint8_t* kernel_id, int on_dev)
{
    if (!st || !xi || !attr || !cell_start || !dv) return SDM_EINVAL;
    if (n_sd > st->cap) return SDM_ECAPACITY;
    std::vector<uint64_t> hx;
    std::vector<double> ha, hdv;
    std::vector<uint32_t> hcs;
    std::vector<uint8_t> hk;
    SDM_TRY(to_host(hcs, cell_start, (uint64_t)st->n_cell + 1, on_dev, st->stream));
    if (hcs[0] != 0 || hcs[st->n_cell] != n_sd) return SDM_EINVAL;
    for (uint32_t c = 0; c < st->n_cell; ++c)
        if (hcs[c + 1] < hcs[c]) return SDM_EINVAL;
    SDM_TRY(to_host(hx, xi, n_sd, on_dev, st->stream));
    SDM_TRY(to_host(ha, attr, n_sd * st->n_attr, on_dev, st->stream));
    SDM_TRY(to_host(hdv, dv, st->n_cell, on_dev, st->stream));
    if (kernel_id) SDM_TRY(to_host(hk, kernel_id, st->n_cell, on_dev, st->stream));
    return init_common(st, hx.data(), ha.data(), hcs, n_sd, hdv.data(), kernel_id ? hk.data() : nullptr);
}

sdm_status sdm_set_state(sdm_state* st, const uint64_t* xi, const double* attr, int on_dev)
{
    if (!st || !xi || !attr) return SDM_EINVAL;
    if (!st->initialised) return SDM_EINVAL;
    const uint64_t n = st->n_sd;
    const cudaMemcpyKind k = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    SDM_CUDA(cudaMemcpyAsync(st->d_xi, xi, sizeof(uint64_t) * n, k, st->stream));
    for (uint32_t a = 0; a < st->n_attr; ++a)
        SDM_CUDA(cudaMemcpyAsync(st->d_attr + (uint64_t)a * st->cap, attr + (uint64_t)a * n, sizeof(double) * n, k,
                                 st->stream));
    if (n) {
        const uint32_t grid = (uint32_t)std::min<uint64_t>((n + 255) / 256, 4 * (uint64_t)st->n_sm);
        validate_kernel<<<grid, 256, 0, st->stream>>>(st->d_xi, st->d_attr, n, st->cap, st->n_attr, st->d_cell_start,
                                                      st->n_cell, st->d_err);
        SDM_CUDA(cudaGetLastError());
    }
    if (st->d_big_removed)    // the new state is compact: no large cell awaits compaction
        SDM_CUDA(cudaMemsetAsync(st->d_big_removed, 0, sizeof(uint32_t) * (big_ticket_word(st->n_big) + 2 + BIG_SYNC_WORDS),
                                 st->stream));
    st->big_deferred = false;
    const uint32_t cgrid = std::max<uint32_t>(1, std::min<uint32_t>((st->n_cell + 255) / 256, 4 * st->n_sm));
    live_count_kernel<<<cgrid, 256, 0, st->stream>>>(st->d_xi, st->d_cell_start, st->n_cell, st->d_n_live);
    SDM_CUDA(cudaGetLastError());
    return refresh_big_bounds(st);
}

sdm_status sdm_get_state(sdm_state* st, uint64_t* xi, double* attr, uint32_t* cell_start, uint64_t* n_sd, int on_dev)
{
    if (!st || !st->initialised) return SDM_EINVAL;
    SDM_TRY(flush_big_compaction(st));
    const uint64_t n = st->n_sd;
    const cudaMemcpyKind k = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (xi) SDM_CUDA(cudaMemcpyAsync(xi, st->d_xi, sizeof(uint64_t) * n, k, st->stream));
    if (attr)
        for (uint32_t a = 0; a < st->n_attr; ++a)
            SDM_CUDA(cudaMemcpyAsync(attr + (uint64_t)a * n, st->d_attr + (uint64_t)a * st->cap, sizeof(double) * n, k,
                                     st->stream));
    if (cell_start) {
        if (on_dev)
            SDM_CUDA(cudaMemcpyAsync(cell_start, st->d_cell_start, sizeof(uint32_t) * (st->n_cell + 1),
                                     cudaMemcpyDeviceToDevice, st->stream));
        else
            std::memcpy(cell_start, st->h_cell_start.data(), sizeof(uint32_t) * (st->n_cell + 1));
    }
    if (n_sd) *n_sd = n;
    if (!on_dev) SDM_CUDA(cudaStreamSynchronize(st->stream));
    return SDM_OK;
}

sdm_status sdm_coalescence_step(sdm_state* st, const sdm_step_params* p, uint32_t n_steps, sdm_step_stats* stats)
{
    if (!st || !p) return SDM_EINVAL;
    if (!st->initialised) return SDM_EINVAL;
    if (!(p->dt > 0.0) || !std::isfinite(p->dt)) return SDM_EINVAL;
    if (p->precision > SDM_PREC_SURROGATE) return SDM_EINVAL;
    if (p->precision == SDM_PREC_SURROGATE && (!st->d_surr || p->shuffle != SDM_SHUFFLE_PRP)) return SDM_EINVAL;
    if (p->shuffle > SDM_SHUFFLE_SORT || p->reserved != 0) return SDM_EINVAL;
    if (!(p->golovin_b >= 0.0) || !std::isfinite(p->golovin_b)) return SDM_EINVAL;
    if (!(p->efield >= 0.0 && p->efield <= 1.0)) return SDM_EINVAL;
    if (n_steps == 0) return SDM_OK;
    if (stats) SDM_CUDA(cudaMemsetAsync(st->d_stats, 0, 5 * sizeof(unsigned long long), st->stream));
    SDM_TRY(launch_steps(st, p, n_steps, stats != nullptr));
    if (stats) {
        unsigned long long h[5];
        uint32_t e = 0;
        SDM_CUDA(cudaMemcpyAsync(h, st->d_stats, sizeof h, cudaMemcpyDeviceToHost, st->stream));
        SDM_CUDA(cudaMemcpyAsync(&e, st->d_err, sizeof e, cudaMemcpyDeviceToHost, st->stream));
        SDM_CUDA(cudaStreamSynchronize(st->stream));
        stats->n_pairs = h[0];
        stats->n_collisions = h[1];
        stats->n_removed = h[2];
        stats->sum_gamma = h[3];
        stats->n_fp64 = h[4];
        if (e) {
            SDM_TRY(clear_device_error(st, e));
            return err_to_status(e);
        }
    }
    return SDM_OK;
}

sdm_status sdm_remove_zero(sdm_state* st, uint64_t* n_live)
{
    if (!st || !st->initialised) return SDM_EINVAL;
    if (!n_live) return SDM_OK;
    SDM_TRY(flush_big_compaction(st));
    SDM_CUDA(cudaMemsetAsync(st->d_acc, 0, sizeof(unsigned long long), st->stream));
    if (st->n_sd) {
        const uint32_t grid = (uint32_t)std::min<uint64_t>((st->n_sd + 255) / 256, 4 * (uint64_t)st->n_sm);
        count_live_kernel<<<grid, 256, 0, st->stream>>>(st->d_xi, st->n_sd, st->d_acc);
        SDM_CUDA(cudaGetLastError());
    }
    unsigned long long h = 0;
    SDM_CUDA(cudaMemcpyAsync(&h, st->d_acc, sizeof h, cudaMemcpyDeviceToHost, st->stream));
    SDM_CUDA(cudaStreamSynchronize(st->stream));
    *n_live = h;
    return SDM_OK;
}

sdm_status sdm_check_state(sdm_state* st, uint64_t* n_bad_live, uint64_t* n_bad_key)
{
    if (!st || !st->initialised || !n_bad_live || !n_bad_key) return SDM_EINVAL;
    SDM_TRY(flush_big_compaction(st));
    SDM_CUDA(cudaMemsetAsync(st->d_acc, 0, 2 * sizeof(unsigned long long), st->stream));
    if (st->n_sd) {
        const uint32_t grid = (uint32_t)std::min<uint64_t>((st->n_sd + 255) / 256, 4 * (uint64_t)st->n_sm);
        check_live_kernel<<<grid, 256, 0, st->stream>>>(st->d_xi, st->n_sd, st->d_cell_start, st->n_cell,
                                                        st->d_n_live, st->d_acc);
        SDM_CUDA(cudaGetLastError());
    }
    if (st->n_big) {
        check_keys_kernel<<<st->n_chunks, 256, 0, st->stream>>>(st->d_attr, st->d_vbin, st->d_big, st->d_chunks,
                                                                st->d_acc + 1);
        SDM_CUDA(cudaGetLastError());
    }
    if (st->n_wcells) {
        const uint32_t grid = std::max<uint32_t>(1, std::min<uint32_t>((st->n_wcells + 7) / 8, 8 * st->n_sm));
        check_wcell_keys_kernel<<<grid, 256, 0, st->stream>>>(st->d_xi, st->d_attr, st->d_vbin, st->d_cell_start,
                                                              st->d_wcells, st->n_wcells, st->d_cell_xmax,
                                                              st->d_acc + 1);
        SDM_CUDA(cudaGetLastError());
    }
    unsigned long long h[2] = {0, 0};
    SDM_CUDA(cudaMemcpyAsync(h, st->d_acc, sizeof h, cudaMemcpyDeviceToHost, st->stream));
    SDM_CUDA(cudaStreamSynchronize(st->stream));
    *n_bad_live = h[0];
    *n_bad_key = h[1];
    return SDM_OK;
}

sdm_status sdm_rebucket(sdm_state* st, const uint32_t* cell_id, int ptrs_on_device)
{
    if (!st || !st->initialised || !cell_id) return SDM_EINVAL;
    if (st->ws) return SDM_ENOTSUP;                  // needs scratch beyond a caller's workspace
    const uint64_t n = st->n_sd;
    if (n == 0) return SDM_OK;
    if (n >= (1ull << 32)) return SDM_ENOTSUP;
    SDM_TRY(flush_big_compaction(st));
    cudaStream_t s = st->stream;
    const uint32_t n_tiles = (uint32_t)((n + RB_TILE - 1) / RB_TILE);
    // scratch: cid | key 2 | val 2 | count | first | hist | tot | base | err | xi_new | attr_new
    const size_t b_u32 = sizeof(uint32_t) * (5 * n + 2 * (size_t)st->n_cell + 1 + 256 * (size_t)n_tiles + 512 + 4);
    const size_t b_new = sizeof(uint64_t) * st->cap + sizeof(double) * st->cap * st->n_attr;
    if (st->rb_bytes < b_new + b_u32 + 256) {             // grown on demand, freed by sdm_free
        if (st->rb_buf) {
            SDM_CUDA(cudaStreamSynchronize(s));
            cudaFree(st->rb_buf);
            st->rb_buf = nullptr;
            st->rb_bytes = 0;
        }
        if (cudaMalloc((void**)&st->rb_buf, b_new + b_u32 + 256) != cudaSuccess) {
            cudaGetLastError();
            return SDM_ENOMEM;
        }
        st->rb_bytes = b_new + b_u32 + 256;
    }
    char* buf = st->rb_buf;
    uint64_t* xi_new = (uint64_t*)buf;
    double* attr_new = (double*)(buf + sizeof(uint64_t) * st->cap);
    uint32_t* u = (uint32_t*)(buf + b_new);
    uint32_t* cid = u;
    uint32_t* key0 = cid + n;
    uint32_t* key1 = key0 + n;
    uint32_t* val0 = key1 + n;
    uint32_t* val1 = val0 + n;
    uint32_t* count = val1 + n;
    uint32_t* first = count + st->n_cell;
    uint32_t* hist = first + st->n_cell + 1;
    uint32_t* tot = hist + 256 * (size_t)n_tiles;
    uint32_t* base = tot + 256;
    uint32_t* err = base + 256;
    sdm_status rs = SDM_OK;
    auto fail = [&](sdm_status e) { return e; };
    if (cudaMemcpyAsync(cid, cell_id, sizeof(uint32_t) * n,
                        ptrs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(count, 0, sizeof(uint32_t) * st->n_cell, s) != cudaSuccess ||
        cudaMemsetAsync(err, 0, sizeof(uint32_t), s) != cudaSuccess)
        return fail(SDM_ECUDA);
    const uint32_t grid = (uint32_t)std::min<uint64_t>((n + 255) / 256, 8 * (uint64_t)st->n_sm);
    rb_keys_kernel<<<grid, 256, 0, s>>>(st->d_xi, cid, n, st->n_cell, key0, val0, count, err);
    rb_capacity_kernel<<<std::max<uint32_t>(1, std::min<uint32_t>((st->n_cell + 255) / 256, 4 * st->n_sm)), 256, 0,
                         s>>>(count, st->d_cell_start, st->n_cell, err);
    uint32_t h_err = 0;
    if (cudaMemcpyAsync(&h_err, err, sizeof h_err, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(SDM_ECUDA);
    if (h_err & 1u) return fail(SDM_EINVAL);              // a live SD's index is not a cell
    if (h_err & ERR_CAPACITY) return fail(SDM_ECAPACITY);  // a cell would overflow: state unchanged
    // the stable sort by new cell, 8 bits per pass (the dead slots' key n_cell included)
    const uint32_t bits = std::max<uint32_t>(1, ceil_log2_h((uint64_t)st->n_cell + 1));
    uint32_t *kin = key0, *kout = key1, *vin = val0, *vout = val1;
    for (uint32_t shift = 0; shift < bits; shift += 8) {
        rb_hist_kernel<<<n_tiles, RB_THREADS, 0, s>>>(kin, n, shift, n_tiles, hist);
        rb_scan_rows_kernel<<<256, RB_THREADS, 0, s>>>(hist, n_tiles, tot);
        rb_scan_digits_kernel<<<1, 256, 0, s>>>(tot, base);
        rb_scatter_kernel<<<n_tiles, RB_THREADS, 0, s>>>(kin, vin, n, shift, n_tiles, hist, base, kout, vout);
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    rb_first_kernel<<<1, 1024, 0, s>>>(count, st->n_cell, first);
    if (cudaMemsetAsync(buf, 0, b_new, s) != cudaSuccess) return fail(SDM_ECUDA);
    rb_gather_kernel<<<grid, 256, 0, s>>>(kin, vin, n, st->n_cell, first, st->d_cell_start, st->d_xi, st->d_attr, st->cap,
                                          st->n_attr, xi_new, attr_new);
    if (cudaMemcpyAsync(st->d_xi, xi_new, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return fail(SDM_ECUDA);
    for (uint32_t a = 0; a < st->n_attr; ++a)
        if (cudaMemcpyAsync(st->d_attr + (uint64_t)a * st->cap, attr_new + (uint64_t)a * st->cap, sizeof(double) * n,
                            cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return fail(SDM_ECUDA);
    if (cudaMemcpyAsync(st->d_n_live, count, sizeof(uint32_t) * st->n_cell, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return fail(SDM_ECUDA);
    if (cudaGetLastError() != cudaSuccess) return fail(SDM_ECUDA);
    rs = refresh_big_bounds(st);                           // multiplicity bounds and volume bins
    return rs;
}

sdm_status sdm_totals(sdm_state* st, uint64_t* n_total, double* mass, uint64_t* n_live)
{
    if (!st || !st->initialised) return SDM_EINVAL;
    SDM_TRY(flush_big_compaction(st));
    SDM_CUDA(cudaMemsetAsync(st->d_acc, 0, 4 * sizeof(unsigned long long), st->stream));
    if (st->n_sd) {
        const uint32_t grid = (uint32_t)std::min<uint64_t>((st->n_sd + 255) / 256, 4 * (uint64_t)st->n_sm);
        totals_kernel<<<grid, 256, 0, st->stream>>>(st->d_xi, st->d_attr, st->n_sd, st->d_acc, (double*)(st->d_acc + 1),
                                                     st->d_acc + 2);
        SDM_CUDA(cudaGetLastError());
    }
    unsigned long long h[4];
    SDM_CUDA(cudaMemcpyAsync(h, st->d_acc, sizeof h, cudaMemcpyDeviceToHost, st->stream));
    SDM_CUDA(cudaStreamSynchronize(st->stream));
    if (n_total) *n_total = h[0];
    if (mass) std::memcpy(mass, &h[1], sizeof(double));
    if (n_live) *n_live = h[2];
    return SDM_OK;
}

sdm_status sdm_spectrum(sdm_state* st, const double* r_edges, uint32_t n_bins, uint32_t cell, double* out,
                        int out_on_device)
{
    if (!st || !st->initialised || !r_edges || !out || n_bins == 0) return SDM_EINVAL;
    for (uint32_t b = 0; b < n_bins; ++b)
        if (!(r_edges[b] > 0.0) || !(r_edges[b + 1] > r_edges[b]) || !std::isfinite(r_edges[b + 1]))
            return SDM_EINVAL;
    SDM_TRY(flush_big_compaction(st));
    uint32_t c0 = 0, c1 = st->n_cell;
    if (cell != UINT32_MAX) {
        if (cell >= st->n_cell) return SDM_EINVAL;
        c0 = cell;
        c1 = cell + 1;
    }
    std::vector<double> ve(n_bins + 1), msum(n_bins);
    for (uint32_t b = 0; b <= n_bins; ++b) {
        double t = FOUR_PI_OVER_THREE * r_edges[b];
        t = t * r_edges[b];
        ve[b] = t * r_edges[b];
    }
    // the fixed-point grid of the exact sums (see spectrum_exact_kernel)
    if (!(ve[0] >= 0x1p-1000) || !std::isfinite(ve[n_bins])) return SDM_EINVAL;
    int e_lo = 0, e_hi = 0;
    std::frexp(ve[0], &e_lo);                       // ve[0] in [2^(e_lo-1), 2^e_lo)
    std::frexp(ve[n_bins], &e_hi);                  // ve[n] < 2^e_hi, so a term < 2^(e_hi + 53)
    const int lsb = (e_lo - 1) - 52;
    const uint32_t W = (uint32_t)((e_hi - lsb) >> 5) + 3;
    const size_t smem = sizeof(unsigned long long) * (size_t)n_bins * W;
    if (smem > SPECTRUM_SMEM_MAX) return SDM_EINVAL;   // edges spanning an absurd range of volumes
    SDM_CUDA(cudaFuncSetAttribute(spectrum_exact_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)SPECTRUM_SMEM_MAX));
    double* d_ve = nullptr;
    SDM_CUDA(cudaMallocAsync((void**)&d_ve, sizeof(double) * (n_bins + 1) + smem, st->stream));
    unsigned long long* d_acc = (unsigned long long*)(d_ve + n_bins + 1);
    std::vector<unsigned long long> words((size_t)n_bins * W);
    sdm_status rs = SDM_OK;
    do {
        if (cudaMemcpyAsync(d_ve, ve.data(), sizeof(double) * (n_bins + 1), cudaMemcpyHostToDevice, st->stream) ||
            cudaMemsetAsync(d_acc, 0, smem, st->stream)) { rs = SDM_ECUDA; break; }
        const uint64_t s0 = st->h_cell_start[c0], s1 = st->h_cell_start[c1];
        if (s1 > s0) {
            const uint32_t grid = (uint32_t)std::min<uint64_t>((s1 - s0 + 255) / 256, 2 * (uint64_t)st->n_sm);
            spectrum_exact_kernel<<<grid, 256, smem, st->stream>>>(st->d_xi, st->d_attr, s0, s1, d_ve, n_bins, lsb,
                                                                  W, d_acc);
            if (cudaGetLastError() != cudaSuccess) { rs = SDM_ECUDA; break; }
        }
        if (cudaMemcpyAsync(words.data(), d_acc, smem, cudaMemcpyDeviceToHost, st->stream) ||
            cudaStreamSynchronize(st->stream)) { rs = SDM_ECUDA; break; }
    } while (0);
    cudaFreeAsync(d_ve, st->stream);
    if (rs != SDM_OK) return rs;
    for (uint32_t b = 0; b < n_bins; ++b) msum[b] = exact_words_to_double(&words[(size_t)b * W], W, lsb);
    double V = 0.0;
    for (uint32_t c = c0; c < c1; ++c) V = V + st->h_dv[c];
    std::vector<double> res(n_bins);
    for (uint32_t b = 0; b < n_bins; ++b) {
        const double dlnr = std::log(r_edges[b + 1]) - std::log(r_edges[b]);
        res[b] = RHO_WATER * msum[b] / (V * dlnr);
    }
    if (out_on_device) {
        SDM_CUDA(cudaMemcpyAsync(out, res.data(), sizeof(double) * n_bins, cudaMemcpyHostToDevice, st->stream));
        SDM_CUDA(cudaStreamSynchronize(st->stream));
    } else {
        std::memcpy(out, res.data(), sizeof(double) * n_bins);
    }
    return SDM_OK;
}

sdm_status sdm_get_schedule(sdm_state* st, sdm_schedule* out)
{
    if (!st || !out) return SDM_EINVAL;
    *out = st->sched;
    return SDM_OK;
}

sdm_status sdm_set_schedule(sdm_state* st, const sdm_schedule* s)
{
    if (!st || !s) return SDM_EINVAL;
    SDM_TRY(check_schedule(*s));
    if (st->initialised) SDM_TRY(flush_big_compaction(st));   // the flags live in the layout
    const sdm_schedule old = st->sched;
    st->sched = *s;
    if (st->initialised) {
        sdm_status r = build_layout(st);
        if (r != SDM_OK) {
            st->sched = old;
            build_layout(st);
            refresh_big_bounds(st);
            return r;
        }
        SDM_TRY(refresh_big_bounds(st));
    }
    return SDM_OK;
}

sdm_status sdm_autotune(sdm_state* st, const sdm_step_params* p, uint32_t n_steps, sdm_schedule* best)
{
    if (!st || !p || !st->initialised || n_steps == 0) return SDM_EINVAL;
    SDM_TRY(flush_big_compaction(st));
    const uint64_t n = st->n_sd;
    // save the state so that every trial starts from it
    uint64_t* sx = nullptr;
    double* sa = nullptr;
    SDM_CUDA(cudaMalloc(&sx, sizeof(uint64_t) * (n + 1)));
    if (cudaMalloc(&sa, sizeof(double) * (n * st->n_attr + 1)) != cudaSuccess) { cudaFree(sx); return SDM_ENOMEM; }
    sdm_status rs = sdm_get_state(st, sx, sa, nullptr, nullptr, 1);
    std::vector<sdm_schedule> cands;
    const sdm_schedule cur = st->sched;
    for (uint32_t ts : {512u, 1024u, 2048u, 4096u})
        for (uint32_t th : {128u, 256u, 512u})
            for (uint32_t pers : {0u, 4u})
                cands.push_back(sdm_schedule{ts, th, cur.bucket_target, pers});
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    sdm_schedule bs = cur;
    float bt = 1e30f;
    auto trial = [&](const sdm_schedule& c) -> float {
        if (sdm_set_schedule(st, &c) != SDM_OK) return 1e30f;
        sdm_step_params q = *p;
        q.d_step = nullptr;
        if (sdm_set_state(st, sx, sa, 1) != SDM_OK) return 1e30f;
        launch_steps(st, &q, 1, false);   // warm-up
        sdm_set_state(st, sx, sa, 1);
        cudaEventRecord(e0, st->stream);
        launch_steps(st, &q, n_steps, false);
        cudaEventRecord(e1, st->stream);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    for (const auto& c : cands) {
        const float t = trial(c);
        if (t < bt) { bt = t; bs = c; }
    }
    // then the bucket width of the large-cell path
    for (uint32_t bw : {128u, 256u, 512u, 1024u}) {
        sdm_schedule c = bs;
        c.bucket_target = bw;
        const float t = trial(c);
        if (t < bt) { bt = t; bs = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rs == SDM_OK) rs = sdm_set_schedule(st, &bs);
    if (rs == SDM_OK) rs = sdm_set_state(st, sx, sa, 1);
    if (rs == SDM_OK) rs = cuda_status(cudaStreamSynchronize(st->stream));
    cudaMemsetAsync(st->d_err, 0, sizeof(uint32_t), st->stream);
    cudaStreamSynchronize(st->stream);
    cudaFree(sx);
    cudaFree(sa);
    if (best) *best = bs;
    return rs;
}

sdm_status sdm_sync(sdm_state* st)
{
    if (!st) return SDM_EINVAL;
    uint32_t e = 0;
    SDM_CUDA(cudaMemcpyAsync(&e, st->d_err, sizeof e, cudaMemcpyDeviceToHost, st->stream));
    SDM_CUDA(cudaStreamSynchronize(st->stream));
    if (e) {
        SDM_TRY(clear_device_error(st, e));
        SDM_CUDA(cudaStreamSynchronize(st->stream));
        return err_to_status(e);
    }
    return SDM_OK;
}

// The self-test's barrier words are words 8 and 9 of the state's 64-byte error block (word 0 is
// the error word; the others are unused).
sdm_status sdm_debug_wait_timeout(sdm_state* st, uint32_t spin_limit, int withhold)
{
    if (!st || spin_limit == 0) return SDM_EINVAL;
    uint32_t* words = st->d_err + 8;
    SDM_CUDA(cudaMemsetAsync(words, 0, 2 * sizeof(uint32_t), st->stream));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(4);
    cfg.blockDim = dim3(32);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    SDM_CUDA(cudaLaunchKernelEx(&cfg, barrier_selftest_kernel, words, words + 1, st->d_err, spin_limit,
                                (uint32_t)(withhold != 0)));
    return SDM_OK;
}

sdm_status sdm_debug_stage_shortfall(sdm_state* st, uint32_t extra_bytes, uint32_t wait_log2)
{
    if (!st || extra_bytes > 4096 || (wait_log2 != 0 && (wait_log2 < 10 || wait_log2 > 31))) return SDM_EINVAL;
    st->dbg_stage_extra = extra_bytes;
    st->dbg_wait_log2 = wait_log2;
    return SDM_OK;
}

sdm_status sdm_debug_bucket_capacity(sdm_state* st, uint32_t cap)
{
    if (!st || !st->initialised || cap < 32 || (cap & 31u) || cap > st->bucket_cap) return SDM_EINVAL;
    st->bucket_cap = cap;
    st->fin_L.cap = cap;
    return SDM_OK;
}

sdm_status sdm_set_profiling(sdm_state* st, int enable)
{
    if (!st) return SDM_EINVAL;
    collect_profile(st);
    st->profiling = enable != 0;
    for (int k = 0; k < SDM_N_KERNEL_KINDS; ++k) { st->prof_launches[k] = 0; st->prof_ms[k] = 0.0; }
    return SDM_OK;
}

sdm_status sdm_get_profile(sdm_state* st, uint32_t* launches, double* ms)
{
    if (!st) return SDM_EINVAL;
    collect_profile(st);
    for (int k = 0; k < SDM_N_KERNEL_KINDS; ++k) {
        if (launches) launches[k] = st->prof_launches[k];
        if (ms) ms[k] = st->prof_ms[k];
    }
    return SDM_OK;
}

sdm_status sdm_launches_per_step(sdm_state* st, uint32_t shuffle, uint32_t* n)
{
    if (!st || !n || shuffle > SDM_SHUFFLE_SORT) return SDM_EINVAL;
    // small cells: one kernel per kind; large cells: one kernel (PRP contract; it compacts the
    // cells the previous step left flagged) or scatter + finish (SORT contract)
    // small cells: one kernel per kind; large cells: one kernel (PRP contract) or scatter + finish
    // (SORT contract); the queue's pair and compaction kernels once when any kernel fills it
    const bool queue = st->n_wcells || (st->n_big && (shuffle == SDM_SHUFFLE_SORT || st->prp_gq));
    *n = (st->n_wcells ? 1u : 0u) + (st->n_tiles ? 1u : 0u) + (queue ? 2u : 0u) +
         (st->n_big ? (shuffle == SDM_SHUFFLE_PRP ? 1u : 2u) : 0u);
    return SDM_OK;
}

sdm_status sdm_eval_pairs(sdm_state* st, uint32_t kernel_id, const double* v1, const double* v2, const uint64_t* xi1,
                          const uint64_t* xi2, uint64_t n, uint32_t n_cell_sd, double dv, double dt, double golovin_b,
                          double efield, double* p64, float* p32, float* err32, double* plite, double* errlite,
                          float* pup)
{
    if (!st || !v1 || !v2 || !xi1 || !xi2 || !p64 || !p32 || !err32) return SDM_EINVAL;
    if (kernel_id > SDM_KERNEL_ELECTRIC || n_cell_sd < 2 || !(dv > 0) || !(dt > 0)) return SDM_EINVAL;
    if (!(efield >= 0.0 && efield <= 1.0)) return SDM_EINVAL;
    if (n == 0) return SDM_OK;
    const uint32_t grid = (uint32_t)std::min<uint64_t>((n + 255) / 256, 8 * (uint64_t)st->n_sm);
    if ((plite == nullptr) != (errlite == nullptr)) return SDM_EINVAL;
    eval_pairs_kernel<<<grid, 256, 0, st->stream>>>(kernel_id, v1, v2, xi1, xi2, n, n_cell_sd, dv, dt, golovin_b,
                                                    efield, p64, p32, err32, plite, errlite, pup);
    SDM_CUDA(cudaGetLastError());
    return SDM_OK;
}

}  // extern "C"
// ---------------------------------------------------------------------------
// Allocation-free single-box step: the large-cell kernels run on the caller's
// arrays with their scratch in a fixed array compiled into the library.
// ---------------------------------------------------------------------------
namespace {

constexpr uint32_t NA_TARGET_BITS = 8;                                    // 256 SDs per bucket on average
constexpr uint32_t NA_MAX_BUCKETS = SDM_NOALLOC_MAX_SD >> NA_TARGET_BITS; // 1024
constexpr uint32_t NA_MAX_CAP = 448;     // bucket_capacity(256): mean 256 + 160 + 32 records
constexpr uint32_t NA_MAX_CHUNKS = (SDM_NOALLOC_MAX_SD + BIG_CHUNK - 1) / BIG_CHUNK;
// byte offsets inside the scratch array
constexpr size_t NA_OFF_CELL = 0;        // BigCell
constexpr size_t NA_OFF_DV = 64;         // double dv
constexpr size_t NA_OFF_KID = 72;        // uint8 kernel id
constexpr size_t NA_OFF_ERR = 128;       // uint32 error word
constexpr size_t NA_OFF_LIVE = 136;      // uint32 cell_start[2], n_live, removal flag, end-of-step ticket, sync words
constexpr size_t NA_OFF_XMAX = 192;      // uint64 largest multiplicity of the box
constexpr size_t NA_OFF_CHUNKS = 256;
constexpr size_t NA_OFF_BBIG = NA_OFF_CHUNKS + sizeof(BigChunk) * NA_MAX_CHUNKS;
constexpr size_t NA_OFF_CURSOR = (NA_OFF_BBIG + sizeof(BucketDesc) * NA_MAX_BUCKETS + 255) / 256 * 256;  // cursors, ticket
constexpr size_t NA_BOOK_WORDS = (size_t)NA_MAX_BUCKETS + 1;
constexpr size_t NA_OFF_PLAN = (NA_OFF_CURSOR + 4 * NA_BOOK_WORDS + 255) / 256 * 256;          // uint4 per bucket
constexpr size_t NA_OFF_RECORDS = (NA_OFF_PLAN + sizeof(uint4) * NA_MAX_BUCKETS + 255) / 256 * 256;
constexpr size_t NA_BYTES = NA_OFF_RECORDS + sizeof(uint64_t) * (size_t)NA_MAX_BUCKETS * NA_MAX_CAP;
static_assert(NA_OFF_RECORDS % 256 == 0, "bulk copies read the records from 16-byte aligned rows");

// one per loaded library and device; its contents persist between calls
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// Device address of the scratch array in the current device's context, looked up on every call
// (a context created after cudaDeviceReset holds the array at a new address), after the
// per-context set-up of the bound table and the shared-memory limits.
sdm_status noalloc_scratch(unsigned char** out)
{
    SDM_TRY(ensure_device_tables());
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return SDM_ECUDA;
    *out = (unsigned char*)p;
    return SDM_OK;
}

}  // namespace

extern "C" sdm_status sdm_coalescence_step_noalloc(uint64_t* xi, double* attr, uint32_t n_attr,
                                                   uint64_t attr_stride, uint32_t n_sd, double dv,
                                                   uint32_t kernel_id, const sdm_step_params* p,
                                                   void* cuda_stream)
{
    if (!p || (n_sd && (!xi || !attr)) || n_attr == 0 || attr_stride < n_sd) return SDM_EINVAL;
    if (n_sd > SDM_NOALLOC_MAX_SD) return SDM_ECAPACITY;
    if (kernel_id > SDM_KERNEL_ELECTRIC || !(dv > 0.0) || !std::isfinite(dv)) return SDM_EINVAL;
    if (!(p->dt > 0.0) || !std::isfinite(p->dt) || p->precision > SDM_PREC_FP32) return SDM_EINVAL;
    if (p->shuffle > SDM_SHUFFLE_SORT || p->reserved != 0) return SDM_EINVAL;
    if (!(p->golovin_b >= 0.0) || !std::isfinite(p->golovin_b)) return SDM_EINVAL;
    if (!(p->efield >= 0.0 && p->efield <= 1.0)) return SDM_EINVAL;
    if (n_sd < 2) return SDM_OK;
    unsigned char* base = nullptr;
    SDM_TRY(noalloc_scratch(&base));
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    // the same geometry as the large-cell path with a 256-SD bucket target
    BigCell C{};
    C.cell = 0;
    C.slot_begin = 0;
    C.width = n_sd;
    C.nbits = ceil_log2_h(n_sd) > NA_TARGET_BITS ? ceil_log2_h(n_sd) - NA_TARGET_BITS : 0;
    C.bucket_base = 0;
    const uint32_t nb = 1u << C.nbits;
    const uint32_t cap = bucket_capacity((n_sd + nb - 1) / nb);
    if (cap > NA_MAX_CAP) return SDM_ECAPACITY;      // not reached: at most 256 SDs per bucket on average
    BigChunk chunks[NA_MAX_CHUNKS];
    uint32_t n_chunks = 0;
    const uint32_t n_of_cell = (n_sd + BIG_CHUNK - 1) / BIG_CHUNK;
    for (uint32_t l = 0; l < n_sd; l += BIG_CHUNK)
        chunks[n_chunks++] = BigChunk{0, l, std::min(n_sd, l + BIG_CHUNK), n_of_cell};
    C.quad_begin = 0;
    const uint32_t n_quads = (n_sd / 2 + 1) / 2;
    BucketDesc bucket_desc[NA_MAX_BUCKETS];
    unsigned char head[256] = {};
    const uint8_t kid = (uint8_t)kernel_id;
    const uint32_t cell_start[2] = {0, n_sd};
    std::memcpy(head + NA_OFF_CELL, &C, sizeof C);
    std::memcpy(head + NA_OFF_DV, &dv, sizeof dv);
    std::memcpy(head + NA_OFF_KID, &kid, 1);
    std::memcpy(head + NA_OFF_LIVE, cell_start, sizeof cell_start);   // n_live, flag and ticket stay 0

    // descriptors in; cursors, tickets, flags and the error word start at zero on every call
    SDM_CUDA(cudaMemcpyAsync(base, head, sizeof head, cudaMemcpyHostToDevice, stream));
    SDM_CUDA(cudaMemcpyAsync(base + NA_OFF_CHUNKS, chunks, sizeof(BigChunk) * n_chunks, cudaMemcpyHostToDevice, stream));
    for (uint32_t k = 0; k < nb; ++k) bucket_desc[k] = BucketDesc{0, 0, 0, C.nbits, 0, 0, 0, 0};
    SDM_CUDA(cudaMemcpyAsync(base + NA_OFF_BBIG, bucket_desc, sizeof(BucketDesc) * nb, cudaMemcpyHostToDevice,
                             stream));
    SDM_CUDA(cudaMemsetAsync(base + NA_OFF_CURSOR, 0, 4 * (NA_MAX_BUCKETS + 1), stream));   // cursors and ticket
    // [0..1] cell_start, [2] n_live, [3] flag, [4..5] 64-bit ticket, [6..13] the PRP sync words
    uint32_t* live = (uint32_t*)(base + NA_OFF_LIVE);
    static_assert(NA_OFF_LIVE + 4 * (6 + BIG_SYNC_WORDS) <= NA_OFF_XMAX, "sync words overlap the bound");
    live_count_kernel<<<1, 32, 0, stream>>>(xi, live, 1, live + 2);
    unsigned long long* d_xmax = (unsigned long long*)(base + NA_OFF_XMAX);      // the early exit's bound
    SDM_CUDA(cudaMemsetAsync(d_xmax, 0, sizeof(unsigned long long), stream));
    big_xmax_kernel<<<n_chunks, 256, 0, stream>>>(xi, attr, nullptr, (const BigCell*)(base + NA_OFF_CELL),
                                                  (const BigChunk*)(base + NA_OFF_CHUNKS), d_xmax);

    StepArgs a{};
    a.xi = xi;
    a.attr = attr;
    a.stride = attr_stride;
    a.n_attr = n_attr;
    a.precision = p->precision;
    a.cell_start = live;
    a.dv = (const double*)(base + NA_OFF_DV);
    a.kid = (const uint8_t*)(base + NA_OFF_KID);
    a.dt = p->dt;
    a.golovin_b = p->golovin_b;
    a.dt_f = (float)p->dt;
    a.golovin_bf = (float)p->golovin_b;
    a.efield = p->efield;
    a.efield_f = (float)p->efield;
    a.seed_lo = (uint32_t)(p->seed & 0xffffffffu);
    a.seed_hi = (uint32_t)(p->seed >> 32);
    a.pk = philox_keys_host(a.seed_lo, a.seed_hi);
    a.step = p->step;
    a.shuffle = p->shuffle;
    a.d_step = p->d_step;
    a.n_live = live + 2;
    a.stats = nullptr;
    a.err = (uint32_t*)(base + NA_OFF_ERR);
    const BigCell* d_cell = (const BigCell*)(base + NA_OFF_CELL);
    const BigBook bb{(unsigned long long*)(live + 4), live + 3, 1, live + 6};
    if (p->shuffle == SDM_SHUFFLE_PRP) {
        int dev = 0, n_sm = 148;
        SDM_CUDA(cudaGetDevice(&dev));
        SDM_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
        BigLaunch L{1, n_quads, d_cell, d_xmax, nullptr, {}};
        L.pc[0] = C;
        big_prp_kernel<false, PRP_THREADS, false><<<prp_grid_size(n_quads, n_sm, PRP_THREADS), PRP_THREADS, 0, stream>>>(
            a, L, bb, WcQueue{});
        SDM_TRY(launch_big_compact(a, d_cell, live + 3, 1, live + 6, n_sm, stream));
    } else {
        uint32_t* cursor = (uint32_t*)(base + NA_OFF_CURSOR);
        // cursors [NA_MAX_BUCKETS], ticket [1]; the plan; the records
        const BucketBook bk{cursor, (uint4*)(base + NA_OFF_PLAN), cursor + NA_MAX_BUCKETS, nb, cap};
        uint64_t* rec = (uint64_t*)(base + NA_OFF_RECORDS);
        const FinishLayout fl = finish_layout(cap, FINISH_SMEM_WAVE, false);   // at most 1024 buckets: one wave
        const uint32_t scatter_smem = sizeof(uint32_t) * 2 * nb;
        big_scatter_kernel<<<n_chunks, BIG_SCATTER_THREADS, scatter_smem, stream>>>(
            a, d_cell, (const BigChunk*)(base + NA_OFF_CHUNKS), rec, bk);
        big_finish_kernel<2, false><<<(nb + fl.warps - 1) / fl.warps, 32 * fl.warps, fl.bytes, stream>>>(
            a, d_cell, (const BucketDesc*)(base + NA_OFF_BBIG), rec, bk.plan, nb, d_xmax, fl, bb, WcQueue{});
    }
    if (p->d_step) advance_step_kernel<<<1, 32, 0, stream>>>(p->d_step, 1u);
    SDM_CUDA(cudaGetLastError());
    uint32_t e = 0;
    SDM_CUDA(cudaMemcpyAsync(&e, base + NA_OFF_ERR, sizeof e, cudaMemcpyDeviceToHost, stream));
    SDM_CUDA(cudaStreamSynchronize(stream));
    return err_to_status(e);
}

// ---------------------------------------------------------------------------
// Learned surrogate of the gravitational kernel
// ---------------------------------------------------------------------------
namespace {

constexpr uint32_t SURR_STAT_N = 65536;

size_t surr_pass_smem() { return sizeof(sdm::SurrSmem); }

// initial weights: uniform in +-sqrt(6 / (fan_in + fan_out)) (Glorot), biases 0, from a
// host Philox stream (purpose 4) so that a seed fixes the whole training
void surr_init_weights(std::vector<float>& w, uint64_t seed)
{
    w.assign(sdm::SURR_NPARAM, 0.0f);
    uint32_t ctr = 0;
    auto u01 = [&]() {
        // Philox4x32-10 on the host (same published algorithm as the device code)
        uint32_t c0 = ctr++, c1 = 0, c2 = 0, c3 = 4u, k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
        for (int r = 0; r < 10; ++r) {
            if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
            const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
            const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0, n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
            c0 = n0; c1 = (uint32_t)p1; c2 = n2; c3 = (uint32_t)p0;
        }
        return ((c0 >> 8) + 0.5) * 0x1p-24;
    };
    auto fill = [&](int off, int n, int fan_in, int fan_out) {
        const double a = std::sqrt(6.0 / (fan_in + fan_out));
        for (int i = 0; i < n; ++i) w[off + i] = (float)(a * (2.0 * u01() - 1.0));
    };
    fill(sdm::SURR_W1, 2 * sdm::SURR_H, 2, sdm::SURR_H);
    fill(sdm::SURR_W2, sdm::SURR_H * sdm::SURR_H, sdm::SURR_H, sdm::SURR_H);
    fill(sdm::SURR_W3, sdm::SURR_H * sdm::SURR_H, sdm::SURR_H, sdm::SURR_H);
    fill(sdm::SURR_W4, sdm::SURR_H, sdm::SURR_H, 1);
}

sdm_status surr_check(const sdm_surrogate* s)
{
    if (!s) return SDM_EINVAL;
    int dev = -1;
    SDM_CUDA(cudaGetDevice(&dev));
    return dev == s->device ? SDM_OK : SDM_EINVAL;
}

}  // namespace

extern "C" {

sdm_status sdm_surrogate_create(sdm_surrogate** out, const sdm_surrogate_params* p, void* cuda_stream)
{
    using namespace sdm;
    if (!out) return SDM_EINVAL;
    *out = nullptr;
    if (!p || p->n_train == 0 || !(p->r_min > 0.0) || !(p->r_max > p->r_min) || !std::isfinite(p->r_max))
        return SDM_EINVAL;
    sdm_surrogate* s = new (std::nothrow) sdm_surrogate();
    if (!s) return SDM_ENOMEM;
    s->stream = (cudaStream_t)cuda_stream;
    s->r_min = p->r_min;
    s->r_max = p->r_max;
    sdm_status st = SDM_OK;
    double* d_K = nullptr;
    do {
        if (cudaGetDevice(&s->device) != cudaSuccess) { st = SDM_ECUDA; break; }
        const size_t nb = sizeof(float) * (5 * (size_t)SURR_NPS + 4);
        if (cudaMalloc(&s->buf, nb) != cudaSuccess ||
            cudaMalloc(&s->mask, SURR_TILES * SURR_TILES) != cudaSuccess ||
            cudaMalloc(&s->tile_err, sizeof(float) * SURR_TILES * SURR_TILES) != cudaSuccess ||
            cudaMalloc(&d_K, sizeof(double) * SURR_STAT_N) != cudaSuccess) {
            cudaGetLastError();
            st = SDM_ENOMEM;
            break;
        }
        if (cudaMemsetAsync(s->buf, 0, nb, s->stream) != cudaSuccess ||
            cudaMemsetAsync(s->mask, 0, SURR_TILES * SURR_TILES, s->stream) != cudaSuccess) { st = SDM_ECUDA; break; }
        SurrTrainArgs& A = s->args;
        A.w32 = s->buf;
        A.wbf = A.w32 + SURR_NPS;       // each array 16-byte aligned (vector loads of the weights)
        A.grad = A.wbf + SURR_NPS;
        A.m = A.grad + SURR_NPS;
        A.v = A.m + SURR_NPS;
        A.loss = A.v + SURR_NPS;
        A.seed_lo = (uint32_t)(p->seed & 0xffffffffu);
        A.seed_hi = (uint32_t)(p->seed >> 32);
        A.ln_rmin = std::log(p->r_min);
        A.ln_rmax = std::log(p->r_max);
        A.c0 = (float)(0.5 * (A.ln_rmin + A.ln_rmax));
        A.c1 = (float)(0.5 * (A.ln_rmax - A.ln_rmin));
        A.n_train = p->n_train;
        A.mu = 0.0f;
        A.sigma = 1.0f;
        A.k_floor = 0.0;
        // target normalisation from the first pairs of the training set
        surr_targets_kernel<<<256, 256, 0, s->stream>>>(A, SURR_STAT_N, d_K);
        std::vector<double> K(SURR_STAT_N);
        if (cudaMemcpyAsync(K.data(), d_K, sizeof(double) * SURR_STAT_N, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
            cudaStreamSynchronize(s->stream) != cudaSuccess) { st = SDM_ECUDA; break; }
        std::vector<double> pos;
        for (double k : K) if (k > 0.0) pos.push_back(k);
        if (pos.empty()) { st = SDM_EINVAL; break; }
        std::nth_element(pos.begin(), pos.begin() + pos.size() / 2, pos.end());
        A.k_floor = 1e-6 * pos[pos.size() / 2];
        double sum = 0.0, sum2 = 0.0;
        for (double k : K) { const double l = std::log(k + A.k_floor); sum += l; sum2 += l * l; }
        const double mean = sum / SURR_STAT_N, var = std::max(sum2 / SURR_STAT_N - mean * mean, 1e-12);
        A.mu = (float)mean;
        A.sigma = (float)std::sqrt(var);
        std::vector<float> w;
        surr_init_weights(w, p->seed);
        if (cudaMemcpyAsync(A.w32, w.data(), sizeof(float) * SURR_NPARAM, cudaMemcpyHostToDevice, s->stream) != cudaSuccess) {
            st = SDM_ECUDA;
            break;
        }
        surr_round_kernel<<<(SURR_NPARAM + 255) / 256, 256, 0, s->stream>>>(A.w32, A.wbf);
        if (cudaFuncSetAttribute(surr_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)surr_pass_smem()) !=
            cudaSuccess) { st = SDM_ECUDA; break; }
        SurrogateDev& D = s->dev;
        D.w = A.wbf;
        D.mask = s->mask;
        D.c0 = A.c0;
        D.c1 = A.c1;
        D.mu = A.mu;
        D.sigma = A.sigma;
        D.k_floor = (float)A.k_floor;
        D.r_min = (float)p->r_min;
        D.r_max = (float)p->r_max;
        if (cudaMalloc(&s->d_dev, sizeof(SurrogateDev)) != cudaSuccess) { cudaGetLastError(); st = SDM_ENOMEM; break; }
        if (cudaMemcpyAsync(s->d_dev, &D, sizeof D, cudaMemcpyHostToDevice, s->stream) != cudaSuccess) { st = SDM_ECUDA; break; }
        if (cudaStreamSynchronize(s->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) st = SDM_ECUDA;
    } while (false);
    if (d_K) cudaFree(d_K);
    if (st != SDM_OK) { sdm_surrogate_free(s); return st; }
    *out = s;
    return SDM_OK;
}

void sdm_surrogate_free(sdm_surrogate* s)
{
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->buf) cudaFree(s->buf);
    if (s->mask) cudaFree(s->mask);
    if (s->tile_err) cudaFree(s->tile_err);
    if (s->d_dev) cudaFree(s->d_dev);
    delete s;
}

sdm_status sdm_surrogate_train(sdm_surrogate* s, uint32_t n_steps, uint32_t batch, float lr, float* loss)
{
    using namespace sdm;
    SDM_TRY(surr_check(s));
    if (batch == 0 || batch % SURR_TB != 0 || !(lr > 0.0f)) return SDM_EINVAL;
    SurrTrainArgs& A = s->args;
    std::vector<float> hl(n_steps, 0.0f);
    float* d_loss_hist = nullptr;
    if (n_steps && cudaMalloc(&d_loss_hist, sizeof(float) * n_steps) != cudaSuccess) { cudaGetLastError(); return SDM_ENOMEM; }
    sdm_status st = SDM_OK;
    for (uint32_t k = 0; k < n_steps && st == SDM_OK; ++k) {
        const double frac = n_steps > 1 ? (double)k / (n_steps - 1) : 0.0;
        const float lr_k = (float)(lr * (0.05 + 0.95 * 0.5 * (1.0 + std::cos(3.141592653589793 * frac))));
        const uint64_t first = (uint64_t)s->steps_done * batch;
        if (cudaMemsetAsync(A.loss, 0, sizeof(float), s->stream) != cudaSuccess) { st = SDM_ECUDA; break; }
        surr_pass_kernel<<<batch / SURR_TB, SURR_THREADS, surr_pass_smem(), s->stream>>>(A, first, batch, nullptr,
                                                                                          nullptr);
        if (cudaMemcpyAsync(d_loss_hist + k, A.loss, sizeof(float), cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess) {
            st = SDM_ECUDA;
            break;
        }
        surr_adam_kernel<<<(SURR_NPARAM + 255) / 256, 256, 0, s->stream>>>(A, lr_k, s->steps_done + 1);
        if (cudaGetLastError() != cudaSuccess) st = SDM_ECUDA;
        ++s->steps_done;
    }
    if (st == SDM_OK && n_steps) {
        if (cudaMemcpyAsync(hl.data(), d_loss_hist, sizeof(float) * n_steps, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
            st = SDM_ECUDA;
    }
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) st = SDM_ECUDA;
    if (d_loss_hist) cudaFree(d_loss_hist);
    if (st == SDM_OK && loss) std::memcpy(loss, hl.data(), sizeof(float) * n_steps);
    return st;
}

sdm_status sdm_surrogate_build_mask(sdm_surrogate* s, float tol, double* frac, float* max_err)
{
    using namespace sdm;
    SDM_TRY(surr_check(s));
    if (!(tol > 0.0f)) return SDM_EINVAL;
    surr_mask_kernel<<<SURR_TILES * SURR_TILES / 16, 256, 0, s->stream>>>(s->dev, s->args.ln_rmin, s->args.ln_rmax, tol,
                                                                            s->mask, s->tile_err);
    SDM_CUDA(cudaGetLastError());
    std::vector<uint8_t> m(SURR_TILES * SURR_TILES);
    std::vector<float> e(SURR_TILES * SURR_TILES);
    SDM_CUDA(cudaMemcpyAsync(m.data(), s->mask, m.size(), cudaMemcpyDeviceToHost, s->stream));
    SDM_CUDA(cudaMemcpyAsync(e.data(), s->tile_err, sizeof(float) * e.size(), cudaMemcpyDeviceToHost, s->stream));
    SDM_CUDA(cudaStreamSynchronize(s->stream));
    if (frac) {
        size_t used = 0, total = 0;
        for (int a = 0; a < SURR_TILES; ++a)
            for (int b = 0; b <= a; ++b) { ++total; used += m[a * SURR_TILES + b]; }
        *frac = (double)used / (double)total;
    }
    if (max_err) std::memcpy(max_err, e.data(), sizeof(float) * e.size());
    return SDM_OK;
}

sdm_status sdm_surrogate_params_io(sdm_surrogate* s, float* host_params, int set)
{
    using namespace sdm;
    SDM_TRY(surr_check(s));
    if (!host_params) return SDM_EINVAL;
    if (set) {
        SDM_CUDA(cudaMemcpyAsync(s->args.w32, host_params, sizeof(float) * SURR_NPARAM, cudaMemcpyHostToDevice, s->stream));
        surr_round_kernel<<<(SURR_NPARAM + 255) / 256, 256, 0, s->stream>>>(s->args.w32, s->args.wbf);
        SDM_CUDA(cudaGetLastError());
    } else {
        SDM_CUDA(cudaMemcpyAsync(host_params, s->args.w32, sizeof(float) * SURR_NPARAM, cudaMemcpyDeviceToHost, s->stream));
    }
    SDM_CUDA(cudaStreamSynchronize(s->stream));
    return SDM_OK;
}

sdm_status sdm_surrogate_info(const sdm_surrogate* s, double* out)
{
    if (!s || !out) return SDM_EINVAL;
    out[0] = s->args.c0;
    out[1] = s->args.c1;
    out[2] = s->args.mu;
    out[3] = s->args.sigma;
    out[4] = s->args.k_floor;
    out[5] = s->r_max / s->r_min;
    return SDM_OK;
}

sdm_status sdm_surrogate_loss_grad(sdm_surrogate* s, const float* x, const float* t, uint64_t n, float* loss,
                                   float* grad)
{
    using namespace sdm;
    SDM_TRY(surr_check(s));
    if (!x || !t || !loss || !grad || n == 0 || n > (1ull << 30)) return SDM_EINVAL;
    SurrTrainArgs A = s->args;
    SDM_CUDA(cudaMemsetAsync(A.grad, 0, sizeof(float) * SURR_NPARAM, s->stream));
    SDM_CUDA(cudaMemsetAsync(A.loss, 0, sizeof(float), s->stream));
    surr_pass_kernel<<<(uint32_t)((n + SURR_TB - 1) / SURR_TB), SURR_THREADS, surr_pass_smem(), s->stream>>>(A, 0, n, x, t);
    SDM_CUDA(cudaGetLastError());
    SDM_CUDA(cudaMemcpyAsync(grad, A.grad, sizeof(float) * SURR_NPARAM, cudaMemcpyDeviceToHost, s->stream));
    SDM_CUDA(cudaMemcpyAsync(loss, A.loss, sizeof(float), cudaMemcpyDeviceToHost, s->stream));
    SDM_CUDA(cudaMemsetAsync(A.grad, 0, sizeof(float) * SURR_NPARAM, s->stream));   // training expects zeros
    SDM_CUDA(cudaStreamSynchronize(s->stream));
    return SDM_OK;
}

sdm_status sdm_surrogate_eval(sdm_surrogate* s, const double* R, const double* r, uint64_t n, float* K)
{
    using namespace sdm;
    SDM_TRY(surr_check(s));
    if (!R || !r || !K) return SDM_EINVAL;
    if (n == 0) return SDM_OK;
    surr_eval_warp_kernel<<<(uint32_t)std::min<uint64_t>((n + 255) / 256, 4096), 256, 0, s->stream>>>(s->dev, R, r, n,
                                                                                                      K);
    SDM_CUDA(cudaGetLastError());
    return SDM_OK;
}

sdm_status sdm_attach_surrogate(sdm_state* st, const sdm_surrogate* s)
{
    if (!st) return SDM_EINVAL;
    if (!s) {
        st->d_surr = nullptr;
        return SDM_OK;
    }
    if (s->device != st->device) return SDM_EINVAL;
    st->d_surr = s->d_dev;
    return SDM_OK;
}

}  // extern "C"
