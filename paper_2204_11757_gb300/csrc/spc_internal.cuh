// Internal declarations of libspcoarsen (GB300, sm_103a).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "../../include/spcoarsen.h"

namespace spc {

constexpr int kThreads = 256;          // default block size
constexpr uint32_t kSpinLimit = 1u << 22;  // default bound of every device-side retry loop

// bits of the device status word
enum : uint32_t {
    DEV_NOT_SYMMETRIC = 1u << 0,
    DEV_SELF_LOOP = 1u << 1,
    DEV_UNSORTED = 1u << 2,
    DEV_BAD_WEIGHT = 1u << 3,
    DEV_TIMEOUT = 1u << 4,
    DEV_OVERFLOW = 1u << 5,
    DEV_TOO_LARGE = 1u << 6,
    DEV_BAD_ARG = 1u << 7,
};

spc_status status_from_bits(uint32_t bits);

#define SPC_CUDA(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            spc::set_last_cuda_error(e_, #call, __FILE__, __LINE__);                     \
            return SPC_ERR_CUDA;                                                         \
        }                                                                                \
    } while (0)

#define SPC_TRY(call)                                                                    \
    do {                                                                                 \
        spc_status s_ = (call);                                                          \
        if (s_ < 0) return s_;                                                           \
    } while (0)

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);

// ---- workspace ------------------------------------------------------------------------------

struct Block {
    void* p = nullptr;
    size_t bytes = 0;
};

struct Context;

// A named, growable device buffer owned by the context.
struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// Device buffers of one level (inputs of the next level live in `out_*`).
struct LevelBufs {
    Buf lift, emap, self_mass, a_und, rowptr_c, col_c, w_c, perm, seg, score, graph_ptr_c;
    // self-mass reading: accumulated internal weight of every super-node of this level
    // (`mass_ptr` is self_mass itself on the first level, else `mass`; null when not carried)
    Buf mass;
    const void* mass_ptr = nullptr;
    int64_t n = 0, m = 0, n_c = 0, m_c = 0, m_inter = 0;
    int32_t status = 0;
    spc_dtype wtype = SPC_F64;
    float ms = -1.f;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

// Device buffers of per-binade prefix tables over a batch of long sequences (spc_seqtab.cu).
struct SeqTabBufs {
    Buf eblo, nE, tsize, tcnt, tab_off, trip_off, P, T, csum, ctie, loff, mn, mx;
    // full sums: units of the terms and their prefix, per-sequence scale, and per (sequence,
    // binade) pair its window of positions, table offset and chunk offset
    Buf units, cunits, gexp, npe, poff, pw0, plen, pnch, pq, pe, ptoff, pcoff;
    int64_t nseq = 0;
};

// Work buffers shared by all levels (sized for level 0).
struct Work {
    Buf up_cnt, up_ptr, first_up, eu, ev, w_und, deg, p;       // S0-S2
    Buf pk;                                                     // binary32 (column, p) pairs
    Buf sym;                                                    // symmetry fingerprint (u64)
    Buf long_rows, lr_base, lr_len, lr_idx, lr_eoff, heavy, seg_base, seg_len, seg_idx, seg_terms;
    Buf hub_leaf;                                               // per hub: its leaf edges' score
    Buf hub_map, hub_slot;                                      // column maps of the largest hubs
    SeqTabBufs tab_w, tab_p, tab_s;                             // long sums: degrees, hubs, segments
    Buf parent, best_k[2], best_e[2], wl_e[2], wl_u[2], wl_v[2], msf;   // S5 MSF
    Buf counters, key_hist;                                     // small device ints
    Buf sel_key, sel_val, sel_key2, sel_val2, node_graph, seg_start, k_graph;  // selection
    Buf g_need, g_tau, g_lo, g_short;                           // per-graph prefixes (batch)
    Buf parent2, flag, ids;                                     // S6
    Buf c_key, c_val, c_key2, c_val2, c_flag, c_pos, c_head, cU, cV;    // S7
    Buf t_key, t_val, t_key2, t_val2, up_deg, low_deg, deg_c, ufirst, lstart;
    Buf i_key, i_val, i_key2, i_val2, long_segs;                // intra edges (self-mass)
    Buf c_item, i_item;                                         // bucket items (16 / 8 bytes)
    Buf lower_long;                                             // count of long lower rows
    // contraction buckets: sizes (zero between calls), offsets, ranking statistics
    Buf b_cnt, b_off, b_stats, b_list;
    bool b_dirty = true;
    Buf sort_hist, scan_tmp;                                    // sort / scan temporaries
    Buf stage_rowptr, stage_col, stage_w, stage_lift, stage_gptr;  // host staging
    Buf pool_key, pool_val, pool_key2, pool_val2, pool_cnt, pool_off;  // feature pooling
    Buf pool_nch, pool_choff, pool_owner, pool_part;
    // the same temporaries for work running on the second stream (SideBranch)
    Buf sort_hist_side, scan_tmp_side, long_segs_side;
    Buf seg_base_side, seg_len_side, seg_idx_side, seg_terms_side;
    SeqTabBufs tab_s_side;
    Buf lift_final;                                             // composed lift of a call
    // self-mass reading: super-node members sorted by (super-node, id), and the next level's
    // input graph with the accumulated internal weight on its diagonal
    Buf ms_key, ms_val, ms_key2, ms_val2, ms_start;
    Buf dg_rowptr, dg_col, dg_w, dg_pos;
    // adjacency reordering: labels, sort keys, the renumbering and the renumbered CSR
    Buf ro_dist, ro_key, ro_val, ro_key2, ro_val2, ro_perm, ro_deg;
    Buf ro_rowptr, ro_col, ro_w, ro_lkey, ro_lkey2, ro_lval, ro_lval2, ro_head, ro_lift;
};

struct Timer {
    std::string substr;      // kernels whose name contains it are timed; "*" times every kernel
    bool on = false;
    int64_t launches = 0;
    double total_ms = 0.0;
    // algorithmic bytes of the next launch (set by note_bytes just before it, 0: no model)
    double next_bytes = 0.0;
    struct Pending {
        const char* name;
        cudaEvent_t a, b;
        double bytes;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    struct PerKernel {
        std::string name;
        int64_t launches;
        double ms;
        double bytes;
    };
    std::vector<PerKernel> per_kernel;
};

// Recorded schedule for graph replay: every value the host driver reads back from the device
// during a host-driven run is logged; a capture replays the same control flow from the log and
// enqueues a device-side check of each logged value instead of the read.
struct LevelMeta {
    int64_t n = 0, m = 0, n_c = 0, m_c = 0, m_inter = 0;
    int32_t status = 0;
    spc_dtype wtype = SPC_F64;
    const void* mass_ptr = nullptr;
};

struct Replay {
    enum Mode { kDirect = 0, kRecord = 1, kCapture = 2 };
    Mode mode = kDirect;
    std::vector<int64_t> log;
    size_t pos = 0;
    std::vector<int64_t> key;        // the call the log belongs to
    bool recorded = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t graph_kernels = 0;       // kernel nodes in the captured graph
    std::string timer_substr;        // kernels timed inside the captured graph
    std::vector<Timer::Pending> timed;
    std::vector<LevelMeta> metas;
    int64_t n_c_final = 0;
    int32_t warn = 0;
    int32_t* d_mismatch = nullptr;   // set by the checks of a replay
    unsigned long long* d_hash = nullptr;
    unsigned long long hash = 0;     // checksum of the recorded call's input arrays
    cudaStream_t cap_stream = nullptr;
};

}  // namespace spc

struct spc_context {
    cudaStream_t stream = nullptr;
    spc_allocator allocator{};
    bool has_allocator = false;
    int device = 0;
    int num_sms = 0;
    uint32_t* d_status = nullptr;    // device status word
    uint32_t* h_status = nullptr;    // pinned mirror
    int64_t* h_scalars = nullptr;    // pinned readback area
    std::vector<spc::Block> blocks;  // everything allocated, for destroy
    spc::Work work;
    std::vector<spc::LevelBufs> levels;
    int32_t n_levels = 0;
    int32_t replayed_last = 0;       // the last coarsening call was a graph replay
    bool has_result = false;         // lift_final and the levels hold a coarsening result
    int64_t reorder_n = 0;           // the last coarsening renumbered its n nodes (0: it did not)
    spc::Timer timer;
    int64_t launches = 0;
    spc::Replay replay;
    // score-schedule autotuner: (dtype, log2 mean row length, log2 m) -> 1 edge tiles, 2 warp/row
    std::vector<std::pair<int64_t, int>> tuned;
    cudaEvent_t tune_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    uint64_t sym_key[2] = {0, 0};    // key of the symmetry fingerprint, drawn at creation
    // arithmetic counts of the timed score launches: [0..1] edge tiles (adds, subtractions),
    // [2..3] warp per row, [4..5] staged rows
    unsigned long long* d_ops = nullptr;
    // second stream for independent work inside a level (parallel branches of a captured graph)
    cudaStream_t side_stream = nullptr;
    cudaEvent_t branch_ev[2] = {nullptr, nullptr};
};

namespace spc {

// Work that does not depend on what the main stream does next runs on the context's second
// stream: the constructor makes that stream wait for everything enqueued so far and sends the
// following launches there; leave() sends launches back to the main stream; the destructor
// makes the main stream wait for the side's work (also on an early error return).  Inside a
// stream capture this forms two parallel branches of the graph.  Scratch that both streams
// could use at once (the scan and sort temporaries) is used by one branch only.
// true while launches go to the second stream: such work uses the *_side temporaries
inline bool on_side(const spc_context* ctx) {
    return ctx->side_stream != nullptr && ctx->stream == ctx->side_stream;
}

class SideBranch {
public:
    explicit SideBranch(spc_context* ctx);
    ~SideBranch();
    spc_status status() const { return st_; }
    void leave();
private:
    spc_context* ctx_;
    cudaStream_t main_;
    spc_status st_ = SPC_OK;
    bool forked_ = false;
};

// allocation helpers (allocator callback or cudaMalloc)
spc_status ensure(spc_context* ctx, Buf& b, size_t bytes);
// ensure(), and zero the block whenever it is (re)allocated
spc_status ensure_zeroed(spc_context* ctx, Buf& b, size_t bytes);
void free_all(spc_context* ctx);

// launch accounting + optional timing of selected kernels
void before_launch(spc_context* ctx, const char* name);
void after_launch(spc_context* ctx, const char* name);

// Device counters for a kernel's arithmetic count while that kernel is being timed, else null.
unsigned long long* op_counter(spc_context* ctx, const char* kernel_name, int slot);

// Algorithmic DRAM bytes of the next SPC_LAUNCH (the bytes the operation must move at minimum:
// each input read once, each output written once), reported with the kernel's timed launches
// so a roofline fraction can be formed from live timings.
inline void note_bytes(spc_context* ctx, double bytes) { ctx->timer.next_bytes = bytes; }

inline int grid_for(int64_t items, int threads, int max_blocks) {
    int64_t b = (items + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return static_cast<int>(b);
}

// Kernels of the library are launched with programmatic stream serialization: a kernel may
// be scheduled while its predecessor on the stream is still finishing, and waits in
// pdl_wait() -- the first statement of every kernel -- until that predecessor has completed
// and its writes are visible.  This hides the launch gap between dependent kernels (many of a
// coarsening level's kernels are small).  Launched without the attribute, pdl_wait() returns
// at once.
// The device status block of a context: word 0 is the status word (DEV_* bits), word 1 the
// bound of every device-side wait or retry loop (0: kSpinLimit), set by
// spc_context_set_wait_limit.  A wait that reaches the bound gives up and sets DEV_TIMEOUT.
__device__ __forceinline__ uint32_t spin_limit(const uint32_t* status) {
    const uint32_t v = status[1];
    return v ? v : kSpinLimit;
}

__device__ __forceinline__ void pdl_wait() {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
    asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}

// cp.async copies of one 4- or 8-byte element from global into shared memory (sm_80 and
// later), completed by cp_async_wait_all
__device__ __forceinline__ void cp_async_4(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_8(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
template <class T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem) {
    if constexpr (sizeof(T) == 8) cp_async_8(smem, gmem);
    else cp_async_4(smem, gmem);
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// The rows of a tile of consecutive CSR entries [base, end), for kernels that run flat over the
// stored entries: every thread of the block calls it (it synchronises the block).  Two searches
// find the first row r_lo and the last row of the tile; one thread per row then marks the row
// of each of its entries, s_row[j - base] = row - r_lo, or -2 - (row - r_lo) for a row of
// more than `long_row` entries (long_row < 0: no limit).  Returns r_lo.  Rows spanned by a tile are
// visited by that tile alone (neighbouring tiles share at most one row), so the marking is
// O(rows + entries) over the whole array.
__device__ __forceinline__ int64_t csr_last_row_at(const int64_t* __restrict__ rowptr, int64_t lo,
                                                   int64_t hi, int64_t j) {
    while (lo < hi) {  // the last row x in [lo, hi] with rowptr[x] <= j
        const int64_t mid = (lo + hi + 1) >> 1;
        if (rowptr[mid] <= j) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int64_t tile_rows(const int64_t* __restrict__ rowptr, int64_t n,
                                             int64_t base, int64_t end, int64_t long_row,
                                             int32_t* s_row, int64_t* s_rows) {
    if (threadIdx.x < 2)
        s_rows[threadIdx.x] = csr_last_row_at(rowptr, 0, n - 1, threadIdx.x ? end - 1 : base);
    __syncthreads();
    const int64_t r_lo = s_rows[0], r_hi = s_rows[1];
    for (int64_t x = r_lo + threadIdx.x; x <= r_hi; x += blockDim.x) {
        const int64_t r0 = rowptr[x], r1 = rowptr[x + 1];
        const int32_t rel = (int32_t)(x - r_lo);
        const int32_t mark = (long_row >= 0 && r1 - r0 > long_row) ? -2 - rel : rel;
        for (int64_t j = r0 > base ? r0 : base; j < (r1 < end ? r1 : end); ++j)
            s_row[j - base] = mark;
    }
    __syncthreads();
    return r_lo;
}

template <typename... Params, typename... Args>
cudaError_t launch_pdl(cudaStream_t stream, dim3 grid, dim3 block, size_t smem,
                       void (*kernel)(Params...), Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

#define SPC_LAUNCH(ctx, kernel, grid, block, smem, ...)                                   \
    do {                                                                                 \
        spc::before_launch((ctx), #kernel);                                              \
        cudaError_t le_ = spc::launch_pdl((ctx)->stream, dim3(grid), dim3(block), (smem), \
                                          kernel, __VA_ARGS__);                          \
        if (le_ == cudaSuccess) le_ = cudaGetLastError();                                \
        spc::after_launch((ctx), #kernel);                                               \
        if (le_ != cudaSuccess) {                                                        \
            spc::set_last_cuda_error(le_, #kernel, __FILE__, __LINE__);                  \
            return SPC_ERR_CUDA;                                                         \
        }                                                                                \
    } while (0)

// ---- device-wide primitives (spc_scan.cu, spc_sort.cu) -------------------------------------

// Exclusive scan of n int32 values into out[0..n] (out[n] = total).  in and out may alias.
spc_status scan_i32(spc_context* ctx, const int32_t* in, int32_t* out, int64_t n);
// Same for int64 (out int64).
spc_status scan_i64(spc_context* ctx, const int32_t* in, int64_t* out, int64_t n);
// Same for int64 input.
spc_status scan_i64_i64(spc_context* ctx, const int64_t* in, int64_t* out, int64_t n);
// Exclusive scan of 0/1 bytes into int32 positions, out[n] = total.
spc_status scan_flags_u8(spc_context* ctx, const uint8_t* in, int32_t* out, int64_t n);

// Stable LSD radix sort of (key, value) pairs on key bits [0, end_bit).  The sorted result ends
// in (keys, vals); (keys_alt, vals_alt) are scratch of the same size.  `count` is the number of
// valid items (<= capacity).
spc_status radix_sort_u64(spc_context* ctx, uint64_t* keys, uint32_t* vals, uint64_t* keys_alt,
                          uint32_t* vals_alt, int64_t count, int end_bit);
spc_status radix_sort_u32(spc_context* ctx, uint32_t* keys, uint32_t* vals, uint32_t* keys_alt,
                          uint32_t* vals_alt, int64_t count, int end_bit);

// Context-free variants (caller-owned scratch, explicit stream) used by the allocation-free
// entry point in spc_static.cu.
int64_t scan_raw_tmp_elems(int64_t n);
cudaError_t scan_i32_raw(cudaStream_t stream, const int32_t* in, int32_t* out, int64_t n,
                         int32_t* tmp);
int64_t radix_raw_hist_elems(int64_t count);
cudaError_t radix_sort_u64_raw(cudaStream_t stream, uint64_t* keys, uint32_t* vals,
                               uint64_t* keys_alt, uint32_t* vals_alt, int64_t count,
                               int end_bit, int32_t* hist, int32_t* scan_tmp);

// Per-binade prefix tables over nseq long sequences terms[base[q] .. base[q] + len[q])
// (binary32 when f32, else binary64; all pointers device), over every position and the binades
// of a running sum below 8 (the score walks of hub rows, from any start).
spc_status seqtab_build(spc_context* ctx, const void* terms, bool f32, int64_t nseq,
                        const int64_t* base, const int64_t* len, SeqTabBufs& tb);
// out[out_idx[q]] (or out[q]) = the left-to-right sum from zero of sequence q, through tables
// restricted to the positions where the running sum can lie in each binade.
spc_status seqtab_full(spc_context* ctx, const void* terms, bool f32, int64_t nseq,
                       const int64_t* base, const int64_t* len, const int64_t* out_idx, void* out,
                       SeqTabBufs& tb);

// ---- steps (spc_score.cu, spc_merge.cu, spc_contract.cu) ----------------------------------

struct GraphView {
    int64_t n = 0, nnz = 0, m = 0;
    // diagonal entries (x, x) stored in their rows (the self-mass reading's coarse graphs; 0 for
    // a caller's graph, whose self-loops are rejected): nnz = 2 m + ndiag
    int64_t ndiag = 0;
    const int64_t* rowptr = nullptr;
    const int32_t* col = nullptr;
    const void* w = nullptr;
    spc_dtype wtype = SPC_F64;
};

inline bool score_is_f32(spc_dtype wt) { return wt == SPC_F32; }
inline size_t wsize(spc_dtype wt) { return wt == SPC_F64 ? 8 : 4; }
inline size_t accsize(spc_dtype wt) { return wt == SPC_F32 ? 4 : 8; }

// S0-S3.  Fills g.m (host) -- synchronises once.  Scores go to `score` (u64 bits or u32 bits).
spc_status run_score(spc_context* ctx, GraphView& g, bool validate, void* score, int schedule);

// S5-S6 for one graph or a batch.  targets: host value (B == 1) or device int64 per graph.
struct SelectArgs {
    int64_t B = 1;
    const int64_t* d_graph_ptr = nullptr;  // device [B+1] (batched) or null
    const int64_t* d_targets = nullptr;    // device [B] per-graph targets (batched) or null
    int64_t target = 0;                    // single-graph target
};
spc_status run_select(spc_context* ctx, const GraphView& g, const void* score,
                      const SelectArgs& sa, int32_t* lift, uint8_t* merged, int64_t* n_c,
                      int64_t* graph_ptr_c, int32_t* status);

// S7.  Writes into lv's buffers (allocated by the caller through ensure()).
spc_status run_contract(spc_context* ctx, const GraphView& g, const int32_t* lift, int64_t n_c,
                        LevelBufs& lv);

// S4 (stand-alone fitness sort).
spc_status run_sort_fitness(spc_context* ctx, int64_t m, const void* f, bool f32,
                            int32_t* order_out);

spc_status run_contract_forward(spc_context* ctx, const int32_t* perm, const int32_t* seg,
                                int64_t m_c, const void* w_und, spc_dtype wt, void* a_und);

// The self-mass reading of the multilevel driver (the merged node of the proof of Theorem 2).
// mass_out[U] = (the members' masses prev_mass[x], ascending x, summed left to right from 0)
// + self_mass[U]; prev_mass null means all zero (then mass_out is self_mass itself and nothing
// runs: *mass_ptr = self_mass).  Types: int64 for SPC_I32, else the weight type.
spc_status run_carry_mass(spc_context* ctx, int64_t n, const int32_t* lift, int64_t n_c,
                          const void* prev_mass, const void* self_mass, spc_dtype wt,
                          Buf& mass_out, const void** mass_ptr);
// The graph g with entry (x, x) = 2 mass[x] in its ascending-column place for every x with
// mass[x] != 0 (edge ids unchanged); written into the context's dg_* buffers, described by out.
spc_status run_diag_graph(spc_context* ctx, const GraphView& g, const void* mass,
                          GraphView& out);

// Adjacency reordering (spc_reorder.cu): the graph renumbered by (L_8(x), L_2(x), x), L_k(x) the
// smallest node id within k hops of x, into the context's ro_* buffers (work.ro_perm[x] = the new id of node x), and
// out[x] = in[ro_perm[x]] for a lift computed on the renumbered graph.  g must be valid.
spc_status run_reorder(spc_context* ctx, const GraphView& g, GraphView& out);
spc_status run_unpermute(spc_context* ctx, int64_t n, const int32_t* in, int32_t* out);
// S0 row checks only (monotone row pointers, sorted in-range columns, no self-loop, valid
// weights), synchronising to report them: what the renumbering indexes with.
spc_status run_check_rows(spc_context* ctx, const GraphView& g);
spc_status run_pool_forward(spc_context* ctx, int64_t n, const int32_t* lift, int64_t n_c,
                            int64_t F, spc_dtype dt, const void* x, void* xc);
spc_status run_pool_backward(spc_context* ctx, int64_t n, const int32_t* lift, int64_t n_c,
                             int64_t F, spc_dtype dt, const void* grad_xc, void* grad_x);
spc_status run_contract_backward(spc_context* ctx, const int32_t* emap, int64_t m,
                                 const void* grad_a, void* grad_w, spc_dtype wt);

// read the status word (synchronises)
spc_status sync_status(spc_context* ctx);

// A device value the host driver needs (int32 or int64 at `dev`).  Direct and recording runs
// copy it back (synchronising; a recording run logs it); a capture returns the logged value and
// enqueues a check that flags a replay whose device value differs.
spc_status read_vals(spc_context* ctx, int count, const void* const* dev, const int* bytes,
                     int64_t* out);
spc_status read_i32(spc_context* ctx, const int32_t* dev, int64_t* out);
// a work-list count that drives a loop whose kernels read the count from the device: under
// capture only the final (zero) count is checked on the device
spc_status read_loop_count(spc_context* ctx, const int32_t* dev, int64_t* out);
spc_status read_i64(spc_context* ctx, const int64_t* dev, int64_t* out);
// Mid-pipeline status check: synchronises and returns the status (0 during a capture, whose
// status is read after the replay).
spc_status check_status(spc_context* ctx);
inline bool capturing(const spc_context* ctx) { return ctx->replay.mode == Replay::kCapture; }
// record an event (an external event node during a capture)
cudaError_t record_event(spc_context* ctx, cudaEvent_t ev);

}  // namespace spc
