// C ABI of libspcoarsen: context, workspace, host staging, the level driver and the entry
// points declared in include/spcoarsen.h.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <random>

#include "spc_internal.cuh"

namespace spc {

static thread_local char g_cuda_err[512];

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
    snprintf(g_cuda_err, sizeof(g_cuda_err), "%s (%s) at %s:%d: %s", cudaGetErrorName(e), what,
             file, line, cudaGetErrorString(e));
}

spc_status status_from_bits(uint32_t bits) {
    if (bits & DEV_UNSORTED) return SPC_ERR_UNSORTED;
    if (bits & DEV_SELF_LOOP) return SPC_ERR_SELF_LOOP;
    if (bits & DEV_BAD_WEIGHT) return SPC_ERR_BAD_WEIGHT;
    if (bits & DEV_NOT_SYMMETRIC) return SPC_ERR_NOT_SYMMETRIC;
    if (bits & DEV_TIMEOUT) return SPC_ERR_TIMEOUT;
    if (bits & DEV_OVERFLOW) return SPC_ERR_OVERFLOW;
    if (bits & DEV_TOO_LARGE) return SPC_ERR_TOO_LARGE;
    if (bits & DEV_BAD_ARG) return SPC_ERR_INVALID_ARG;
    return SPC_OK;
}

static spc_status raw_alloc(spc_context* ctx, size_t bytes, void** out) {
    *out = nullptr;
    if (bytes == 0) bytes = 256;
    if (ctx->has_allocator) {
        *out = ctx->allocator.alloc(ctx->allocator.ctx, bytes);
        if (!*out) return SPC_ERR_OOM;
    } else {
        cudaError_t e = cudaMalloc(out, bytes);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            *out = nullptr;
            return SPC_ERR_OOM;
        }
    }
    ctx->blocks.push_back(Block{*out, bytes});
    return SPC_OK;
}

static void raw_free(spc_context* ctx, void* p) {
    if (!p) return;
    for (size_t i = 0; i < ctx->blocks.size(); ++i) {
        if (ctx->blocks[i].p == p) {
            ctx->blocks[i] = ctx->blocks.back();
            ctx->blocks.pop_back();
            break;
        }
    }
    if (ctx->has_allocator) ctx->allocator.free(ctx->allocator.ctx, p);
    else cudaFree(p);
}

spc_status ensure(spc_context* ctx, Buf& b, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    if (b.p && b.bytes >= bytes) return SPC_OK;
    if (capturing(ctx)) return SPC_ERR_CUDA;  // a capture replays a recorded run: no growth
    if (b.p) {
        // the old block may still be read by queued work
        SPC_CUDA(cudaStreamSynchronize(ctx->stream));
        raw_free(ctx, b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    void* p = nullptr;
    SPC_TRY(raw_alloc(ctx, bytes, &p));
    b.p = p;
    b.bytes = bytes;
    return SPC_OK;
}

spc_status ensure_zeroed(spc_context* ctx, Buf& b, size_t bytes) {
    // a new block can land on the old one's address: compare sizes, not pointers
    const size_t had = b.p ? b.bytes : 0;
    SPC_TRY(ensure(ctx, b, bytes));
    if (b.bytes != had) SPC_CUDA(cudaMemsetAsync(b.p, 0, b.bytes, ctx->stream));
    return SPC_OK;
}

void free_all(spc_context* ctx) {
    cudaStreamSynchronize(ctx->stream);
    while (!ctx->blocks.empty()) raw_free(ctx, ctx->blocks.back().p);
}

static bool timed(const Timer& t, const char* name) {
    return t.on && (t.substr == "*" || strstr(name, t.substr.c_str()) != nullptr);
}

cudaError_t record_event(spc_context* ctx, cudaEvent_t ev) {
    if (capturing(ctx)) return cudaEventRecordWithFlags(ev, ctx->stream, cudaEventRecordExternal);
    return cudaEventRecord(ev, ctx->stream);
}

SideBranch::SideBranch(spc_context* ctx) : ctx_(ctx), main_(ctx->stream) {
    cudaError_t e = cudaSuccess;
    if (!ctx->side_stream) e = cudaStreamCreateWithFlags(&ctx->side_stream, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i)
        if (!ctx->branch_ev[i]) e = cudaEventCreateWithFlags(&ctx->branch_ev[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->branch_ev[0], main_);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->side_stream, ctx->branch_ev[0], 0);
    if (e != cudaSuccess) {
        set_last_cuda_error(e, "SideBranch", __FILE__, __LINE__);
        st_ = SPC_ERR_CUDA;
        return;
    }
    forked_ = true;
    ctx->stream = ctx->side_stream;
}

void SideBranch::leave() { ctx_->stream = main_; }

SideBranch::~SideBranch() {
    ctx_->stream = main_;
    if (!forked_) return;
    if (cudaEventRecord(ctx_->branch_ev[1], ctx_->side_stream) == cudaSuccess)
        cudaStreamWaitEvent(main_, ctx_->branch_ev[1], 0);
}

unsigned long long* op_counter(spc_context* ctx, const char* kernel_name, int slot) {
    if (!ctx->d_ops || !timed(ctx->timer, kernel_name)) return nullptr;
    return ctx->d_ops + slot;
}

void before_launch(spc_context* ctx, const char* name) {
    Timer& t = ctx->timer;
    ctx->launches += 1;
    const double bytes = t.next_bytes;
    t.next_bytes = 0.0;
    if (!timed(t, name)) return;
    cudaEvent_t a, b;
    if (t.pool.size() >= 2) {
        a = t.pool.back(); t.pool.pop_back();
        b = t.pool.back(); t.pool.pop_back();
    } else {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    record_event(ctx, a);
    if (capturing(ctx)) ctx->replay.timed.push_back({name, a, b, bytes});
    else t.pending.push_back({name, a, b, bytes});
}

void after_launch(spc_context* ctx, const char* name) {
    Timer& t = ctx->timer;
    if (!timed(t, name)) return;
    if (capturing(ctx)) record_event(ctx, ctx->replay.timed.back().b);
    else record_event(ctx, t.pending.back().b);
}

static void timer_add(Timer& t, const char* name, double ms, double bytes) {
    t.total_ms += ms;
    t.launches += 1;
    for (auto& pk : t.per_kernel) {
        if (pk.name == name) {
            pk.launches += 1;
            pk.ms += ms;
            pk.bytes += bytes;
            return;
        }
    }
    t.per_kernel.push_back({std::string(name), 1, ms, bytes});
}

// in-graph check of up to four logged values (one launch for all values a read took)
struct Expect {
    const void* dev[4];
    long long want[4];
    int bytes[4];
    int count;
};

__global__ void k_expect(Expect x, int32_t* mismatch) {
    spc::pdl_wait();
    const int i = threadIdx.x;
    if (i >= x.count) return;
    const long long got = x.bytes[i] == 8 ? *static_cast<const long long*>(x.dev[i])
                                          : (long long)*static_cast<const int32_t*>(x.dev[i]);
    if (got != x.want[i]) *mismatch = 1;
}

spc_status read_vals(spc_context* ctx, int count, const void* const* dev, const int* bytes,
                     int64_t* out) {
    Replay& R = ctx->replay;
    if (R.mode == Replay::kCapture) {
        for (int i0 = 0; i0 < count; i0 += 4) {
            Expect x{};
            x.count = count - i0 < 4 ? count - i0 : 4;
            for (int i = 0; i < x.count; ++i) {
                if (R.pos >= R.log.size()) return SPC_ERR_CUDA;  // control flow left the record
                out[i0 + i] = R.log[R.pos++];
                x.dev[i] = dev[i0 + i];
                x.bytes[i] = bytes[i0 + i];
                x.want[i] = (long long)out[i0 + i];
            }
            SPC_LAUNCH(ctx, k_expect, 1, 32, 0, x, R.d_mismatch);
        }
        return SPC_OK;
    }
    for (int i = 0; i < count; ++i) {
        SPC_CUDA(cudaMemcpyAsync(ctx->h_scalars + 16 + i, dev[i], bytes[i], cudaMemcpyDeviceToHost,
                                 ctx->stream));
    }
    SPC_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < count; ++i) {
        out[i] = bytes[i] == 8 ? ctx->h_scalars[16 + i]
                               : (int64_t)*reinterpret_cast<int32_t*>(ctx->h_scalars + 16 + i);
        if (R.mode == Replay::kRecord) R.log.push_back(out[i]);
    }
    return SPC_OK;
}

spc_status read_i32(spc_context* ctx, const int32_t* dev, int64_t* out) {
    const void* p = dev;
    const int b = 4;
    return read_vals(ctx, 1, &p, &b, out);
}

spc_status read_loop_count(spc_context* ctx, const int32_t* dev, int64_t* out) {
    Replay& R = ctx->replay;
    if (R.mode == Replay::kCapture) {
        if (R.pos >= R.log.size()) return SPC_ERR_CUDA;
        *out = R.log[R.pos++];
        // only the count that ends the loop is checked: the loop's kernels take the count from
        // the device, so a different intermediate count changes no result
        if (*out == 0) {
            Expect x{};
            x.count = 1;
            x.dev[0] = dev;
            x.bytes[0] = 4;
            x.want[0] = 0;
            SPC_LAUNCH(ctx, k_expect, 1, 32, 0, x, R.d_mismatch);
        }
        return SPC_OK;
    }
    return read_i32(ctx, dev, out);
}

spc_status read_i64(spc_context* ctx, const int64_t* dev, int64_t* out) {
    const void* p = dev;
    const int b = 8;
    return read_vals(ctx, 1, &p, &b, out);
}

spc_status check_status(spc_context* ctx) {
    if (capturing(ctx)) return SPC_OK;
    return sync_status(ctx);
}

spc_status sync_status(spc_context* ctx) {
    SPC_CUDA(cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(uint32_t),
                             cudaMemcpyDeviceToHost, ctx->stream));
    SPC_CUDA(cudaStreamSynchronize(ctx->stream));
    return status_from_bits(*ctx->h_status);
}

// ---- small kernels of the driver ------------------------------------------------------------

// the lifts of up to kComposeMax levels, applied in order
constexpr int kComposeMax = 64;
struct LiftChain {
    const int32_t* lift[kComposeMax];
    int levels;
};

// out[x] = lift_{L-1}[ ... lift_1[lift_0[x]] ... ]: every node's super-node after all levels
__global__ void k_compose_all(int64_t n, LiftChain ch, int32_t* __restrict__ out) {
    spc::pdl_wait();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        int32_t y = ch.lift[0][x];
        for (int l = 1; l < ch.levels; ++l) y = ch.lift[l][y];
        out[x] = y;
    }
}

__global__ void k_compose_emap(int64_t m, const int32_t* __restrict__ next, int32_t* __restrict__ cur) {
    spc::pdl_wait();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = cur[e];
        cur[e] = k >= 0 ? next[k] : -1;
    }
}

template <class KT>
__global__ void k_sort_prep(int64_t m, const KT* __restrict__ f, KT* __restrict__ key,
                            uint32_t* __restrict__ val) {
    spc::pdl_wait();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        key[e] = f[e];
        val[e] = (uint32_t)e;
    }
}

// caller-supplied lift: every value in [0, n_c)
__global__ void k_check_lift(int64_t n, const int32_t* __restrict__ lift, int64_t n_c,
                             uint32_t* status) {
    spc::pdl_wait();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = lift[x];
        if (c < 0 || (int64_t)c >= n_c) atomicOr(status, DEV_BAD_ARG);
    }
}

__global__ void k_targets(int64_t B, const int64_t* __restrict__ graph_ptr, int64_t divisor,
                          int64_t* __restrict__ targets) {
    spc::pdl_wait();
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < B;
         b += (int64_t)gridDim.x * blockDim.x) {
        int64_t t = (graph_ptr[b + 1] - graph_ptr[b]) / divisor;
        targets[b] = t < 1 ? 1 : t;
    }
}

spc_status run_sort_fitness(spc_context* ctx, int64_t m, const void* f, bool f32,
                            int32_t* order_out) {
    Work& W = ctx->work;
    const int gb = grid_for(m, kThreads, ctx->num_sms * 8);
    if (m <= 0) return SPC_OK;
    if (f32) {
        SPC_LAUNCH(ctx, k_sort_prep<uint32_t>, gb, kThreads, 0, m,
                   static_cast<const uint32_t*>(f), W.sel_key.as<uint32_t>(),
                   reinterpret_cast<uint32_t*>(order_out));
        SPC_TRY(radix_sort_u32(ctx, W.sel_key.as<uint32_t>(), reinterpret_cast<uint32_t*>(order_out),
                               W.sel_key2.as<uint32_t>(), W.sel_val2.as<uint32_t>(), m, 31));
    } else {
        SPC_LAUNCH(ctx, k_sort_prep<uint64_t>, gb, kThreads, 0, m,
                   static_cast<const uint64_t*>(f), W.sel_key.as<uint64_t>(),
                   reinterpret_cast<uint32_t*>(order_out));
        SPC_TRY(radix_sort_u64(ctx, W.sel_key.as<uint64_t>(), reinterpret_cast<uint32_t*>(order_out),
                               W.sel_key2.as<uint64_t>(), W.sel_val2.as<uint32_t>(), m, 63));
    }
    return SPC_OK;
}

// ---- workspace sizing -------------------------------------------------------------------------

static spc_status reserve_work(spc_context* ctx, int64_t n, int64_t m, int64_t B) {
    Work& W = ctx->work;
    const size_t N = (size_t)n + 1, M = (size_t)m + 1;
    SPC_TRY(ensure(ctx, W.up_cnt, N * 4));
    SPC_TRY(ensure(ctx, W.up_ptr, (N + 1) * 4));
    SPC_TRY(ensure(ctx, W.first_up, N * 4));
    SPC_TRY(ensure(ctx, W.eu, M * 4));
    SPC_TRY(ensure(ctx, W.ev, M * 4));
    SPC_TRY(ensure(ctx, W.w_und, M * 8));
    SPC_TRY(ensure(ctx, W.deg, N * 8));
    // stored entries of a level's input: 2m, plus one diagonal entry per node under the
    // self-mass reading
    SPC_TRY(ensure(ctx, W.p, (2 * M + N) * 8));
    // binary32 levels also keep every stored entry as one 8-byte (column, p) pair plus one end
    // marker per row, with room for the 16-byte copies that start or end on a neighbour
    SPC_TRY(ensure(ctx, W.pk, (2 * M + 2 * N + 4) * 8));
    SPC_TRY(ensure(ctx, W.sym, 16));
    SPC_TRY(ensure(ctx, W.long_rows, N * 4));
    SPC_TRY(ensure(ctx, W.lr_base, N * 8));
    SPC_TRY(ensure(ctx, W.lr_len, N * 8));
    SPC_TRY(ensure(ctx, W.lr_idx, N * 8));
    SPC_TRY(ensure(ctx, W.lr_eoff, (N + 1) * 8));
    SPC_TRY(ensure(ctx, W.heavy, M * 4));
    SPC_TRY(ensure(ctx, W.hub_leaf, N * 8));
    SPC_TRY(ensure(ctx, W.seg_base, M * 8));
    SPC_TRY(ensure(ctx, W.seg_len, M * 8));
    SPC_TRY(ensure(ctx, W.seg_idx, M * 8));
    SPC_TRY(ensure(ctx, W.seg_terms, M * 8));
    SPC_TRY(ensure(ctx, W.parent, N * 4));
    for (int i = 0; i < 2; ++i) {
        SPC_TRY(ensure(ctx, W.best_k[i], N * 8));
        SPC_TRY(ensure(ctx, W.best_e[i], N * 4));
        SPC_TRY(ensure(ctx, W.wl_e[i], M * 4));
        SPC_TRY(ensure(ctx, W.wl_u[i], M * 4));
        SPC_TRY(ensure(ctx, W.wl_v[i], M * 4));
    }
    SPC_TRY(ensure(ctx, W.msf, M + 16));
    SPC_TRY(ensure(ctx, W.counters, 64 * 4));
    SPC_TRY(ensure(ctx, W.sel_key, M * 8));
    SPC_TRY(ensure(ctx, W.sel_val, M * 4));
    SPC_TRY(ensure(ctx, W.sel_key2, M * 8));
    SPC_TRY(ensure(ctx, W.sel_val2, M * 4));
    SPC_TRY(ensure(ctx, W.node_graph, N * 4));
    SPC_TRY(ensure(ctx, W.seg_start, ((size_t)B + 1) * 4));
    SPC_TRY(ensure(ctx, W.k_graph, ((size_t)B + 1) * 4));
    SPC_TRY(ensure(ctx, W.parent2, N * 4));
    SPC_TRY(ensure(ctx, W.flag, N * 4));
    SPC_TRY(ensure(ctx, W.ids, (N + 1) * 4));
    SPC_TRY(ensure(ctx, W.c_key, M * 8));
    SPC_TRY(ensure(ctx, W.c_item, M * 16));
    SPC_TRY(ensure(ctx, W.lower_long, 16));
    SPC_TRY(ensure(ctx, W.i_item, M * 8));
    SPC_TRY(ensure(ctx, W.c_val, M * 4));
    SPC_TRY(ensure(ctx, W.c_key2, M * 8));
    SPC_TRY(ensure(ctx, W.c_val2, M * 4));
    SPC_TRY(ensure(ctx, W.c_flag, 2 * M + 16));
    SPC_TRY(ensure(ctx, W.c_pos, (M + 1) * 4));
    SPC_TRY(ensure(ctx, W.c_head, (M + 1) * 4));
    SPC_TRY(ensure(ctx, W.cU, M * 4));
    SPC_TRY(ensure(ctx, W.cV, M * 4));
    SPC_TRY(ensure(ctx, W.t_key, M * 4));
    SPC_TRY(ensure(ctx, W.t_val, M * 4));
    SPC_TRY(ensure(ctx, W.t_key2, M * 4));
    SPC_TRY(ensure(ctx, W.t_val2, M * 4));
    SPC_TRY(ensure(ctx, W.up_deg, (N + 1) * 4));
    SPC_TRY(ensure(ctx, W.low_deg, (N + 1) * 4));
    SPC_TRY(ensure(ctx, W.ufirst, (N + 1) * 4));
    SPC_TRY(ensure(ctx, W.lstart, (N + 1) * 4));
    SPC_TRY(ensure(ctx, W.i_key, M * 4));
    SPC_TRY(ensure(ctx, W.i_val, M * 4));
    SPC_TRY(ensure(ctx, W.i_key2, (M + 1) * 4));
    SPC_TRY(ensure(ctx, W.i_val2, (M + 1) * 4));
    SPC_TRY(ensure(ctx, W.long_segs, (M + 1) * 4));
    SPC_TRY(ensure_zeroed(ctx, W.b_cnt, 2 * N * 4));
    SPC_TRY(ensure(ctx, W.b_off, 2 * N * 4));
    SPC_TRY(ensure_zeroed(ctx, W.b_stats, 8 * 8));
    SPC_TRY(ensure(ctx, W.b_list, (2 * (M / 64 + 1) + 16) * 4));  // long-bucket lists
    // scan of up to max(n, m, 256 * tiles) items -> tile sums; radix histograms
    const size_t big = (N > M ? N : M) + 256 * ((M + 4095) / 4096) + 4096;
    // the scans keep their statuses zero between calls; a new block starts zeroed
    SPC_TRY(ensure_zeroed(ctx, W.scan_tmp, (big / 4096 + 4) * 8 + 256));
    // one-sweep sort: 8 passes x (tiles x 256) look-back words + histograms (sorts of up to
    // max(n, m) items: the super-node members of the self-mass reading sort n)
    const size_t NM = N > M ? N : M;
    SPC_TRY(ensure(ctx, W.sort_hist, (8 * 256 * ((NM + 4095) / 4096) + 8 * 512 + 64) * 4));
    return SPC_OK;
}

// the self-mass reading: member sorts, and the next level's input with its diagonal entries
static spc_status reserve_self_mass(spc_context* ctx, int64_t n, int64_t m, spc_dtype wt) {
    Work& W = ctx->work;
    const size_t N = (size_t)n + 1, M = (size_t)m + 1;
    SPC_TRY(ensure(ctx, W.ms_key, N * 4));
    SPC_TRY(ensure(ctx, W.ms_val, N * 4));
    SPC_TRY(ensure(ctx, W.ms_key2, N * 4));
    SPC_TRY(ensure(ctx, W.ms_val2, N * 4));
    SPC_TRY(ensure(ctx, W.ms_start, (N + 1) * 4));
    SPC_TRY(ensure(ctx, W.dg_rowptr, (N + 1) * 8));
    SPC_TRY(ensure(ctx, W.dg_pos, (N + 1) * 4));
    SPC_TRY(ensure(ctx, W.dg_col, (2 * M + N + 1) * 4));
    SPC_TRY(ensure(ctx, W.dg_w, (2 * M + N + 1) * wsize(wt)));
    return SPC_OK;
}

static spc_status reserve_level(spc_context* ctx, LevelBufs& lv, int64_t n, int64_t m,
                                int64_t B) {
    const size_t N = (size_t)n + 1, M = (size_t)m + 1;
    SPC_TRY(ensure(ctx, lv.lift, N * 4));
    SPC_TRY(ensure(ctx, lv.emap, M * 4));
    SPC_TRY(ensure(ctx, lv.self_mass, N * 8));
    SPC_TRY(ensure(ctx, lv.a_und, M * 8));
    SPC_TRY(ensure(ctx, lv.rowptr_c, (N + 1) * 8));
    SPC_TRY(ensure(ctx, lv.col_c, 2 * M * 4));
    SPC_TRY(ensure(ctx, lv.w_c, 2 * M * 8));
    SPC_TRY(ensure(ctx, lv.perm, M * 4));
    SPC_TRY(ensure(ctx, lv.seg, (M + 1) * 4));
    SPC_TRY(ensure(ctx, lv.score, M * 8));
    SPC_TRY(ensure(ctx, lv.graph_ptr_c, ((size_t)B + 2) * 8));
    SPC_TRY(ensure(ctx, lv.mass, N * 8));
    if (!lv.ev0) {
        SPC_CUDA(cudaEventCreate(&lv.ev0));
        SPC_CUDA(cudaEventCreate(&lv.ev1));
    }
    return SPC_OK;
}

// ---- host staging -----------------------------------------------------------------------------

static bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static spc_status stage_in(spc_context* ctx, const void* src, size_t bytes, Buf& buf,
                           const void** out) {
    if (is_device_ptr(src) || bytes == 0) {
        *out = src;
        return SPC_OK;
    }
    SPC_TRY(ensure(ctx, buf, bytes));
    SPC_CUDA(cudaMemcpyAsync(buf.p, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
    *out = buf.p;
    return SPC_OK;
}

static spc_status check_csr(const spc_csr* g) {
    if (!g || g->n < 0 || g->nnz < 0) return SPC_ERR_INVALID_ARG;
    if (g->wtype != SPC_I32 && g->wtype != SPC_F32 && g->wtype != SPC_F64)
        return SPC_ERR_INVALID_ARG;
    if (g->n >= INT32_MAX || g->nnz / 2 >= INT32_MAX) return SPC_ERR_TOO_LARGE;
    if (!g->rowptr || (g->nnz > 0 && (!g->col || !g->w))) return SPC_ERR_INVALID_ARG;
    if (g->nnz & 1) return SPC_ERR_NOT_SYMMETRIC;
    return SPC_OK;
}

static spc_status stage_graph(spc_context* ctx, const spc_csr* g, GraphView& v) {
    Work& W = ctx->work;
    const void* p;
    v.n = g->n;
    v.nnz = g->nnz;
    v.wtype = g->wtype;
    SPC_TRY(stage_in(ctx, g->rowptr, (size_t)(g->n + 1) * 8, W.stage_rowptr, &p));
    v.rowptr = static_cast<const int64_t*>(p);
    SPC_TRY(stage_in(ctx, g->col, (size_t)g->nnz * 4, W.stage_col, &p));
    v.col = static_cast<const int32_t*>(p);
    SPC_TRY(stage_in(ctx, g->w, (size_t)g->nnz * wsize(g->wtype), W.stage_w, &p));
    v.w = p;
    return SPC_OK;
}

// memory handed to the caller (spc_take_result): not recorded among the context's blocks
static void* alloc_owned(spc_context* ctx, size_t bytes) {
    if (bytes == 0) bytes = 256;
    void* p = nullptr;
    if (ctx->has_allocator) return ctx->allocator.alloc(ctx->allocator.ctx, bytes);
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return p;
}

static void free_owned(spc_context* ctx, void* p) {
    if (!p) return;
    if (ctx->has_allocator) ctx->allocator.free(ctx->allocator.ctx, p);
    else cudaFree(p);
}

static spc_status begin_call(spc_context* ctx) {
    if (!ctx) return SPC_ERR_INVALID_ARG;
    SPC_CUDA(cudaSetDevice(ctx->device));
    SPC_CUDA(cudaMemsetAsync(ctx->d_status, 0, sizeof(uint32_t), ctx->stream));
    return SPC_OK;
}

static spc_status copy_out(spc_context* ctx, void* dst, const void* src, size_t bytes) {
    if (bytes == 0 || dst == src) return SPC_OK;
    SPC_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, ctx->stream));
    return SPC_OK;
}

// ---- the level driver --------------------------------------------------------------------------

struct Schedule {
    int32_t levels = 1;
    bool validate = true;
    bool self_mass = true;   // the self-mass reading of the multilevel driver
    bool reorder = false;    // coarsen the graph renumbered by its hop-min labels
    int schedule = 0;
    // single graph
    int64_t n_c = 1;
    // batch
    int64_t B = 1;
    const int64_t* d_graph_ptr = nullptr;  // level-0 graph_ptr on the device
    int64_t ratio = 1;
};


static spc_status run_levels(spc_context* ctx, const GraphView& g0, const Schedule& S,
                             int32_t* lift_total_dev, int64_t* n_c_final, int32_t* warn) {
    const int L = S.levels < 1 ? 1 : S.levels;
    const bool batched = S.d_graph_ptr != nullptr;
    if ((int)ctx->levels.size() < L) ctx->levels.resize(L);
    int64_t* d_targets = nullptr;
    // reserve everything up front (level sizes are bounded by level 0)
    SPC_TRY(reserve_work(ctx, g0.n, g0.nnz / 2, S.B));
    for (int l = 0; l < L; ++l) SPC_TRY(reserve_level(ctx, ctx->levels[l], g0.n, g0.nnz / 2, S.B));
    if (S.self_mass && L > 1) SPC_TRY(reserve_self_mass(ctx, g0.n, g0.nnz / 2, g0.wtype));
    if (batched) {
        SPC_TRY(ensure(ctx, ctx->work.stage_gptr, ((size_t)S.B + 1) * 8 * (L + 1)));
        d_targets = ctx->work.stage_gptr.as<int64_t>();
    }
    const int maxb = ctx->num_sms * 8;
    GraphView cur = g0;
    const int64_t* cur_gptr = S.d_graph_ptr;
    if (S.reorder) {
        // the caller's rows are checked before the renumbering indexes with them; their
        // symmetry is checked by the renumbered graph's first score walk
        if (S.validate) SPC_TRY(run_check_rows(ctx, cur));
        GraphView rg;
        SPC_TRY(run_reorder(ctx, cur, rg));
        cur = rg;
        SPC_TRY(ensure(ctx, ctx->work.ro_lift, ((size_t)g0.n + 1) * 4));
    }
    int32_t* lift_comp = S.reorder ? ctx->work.ro_lift.as<int32_t>() : lift_total_dev;
    const void* mass = nullptr;  // accumulated internal weight of cur's nodes (null: all zero)
    *warn = 0;
    ctx->n_levels = 0;
    for (int l = 0; l < L; ++l) {
        LevelBufs& lv = ctx->levels[l];
        SPC_CUDA(record_event(ctx, lv.ev0));
        SelectArgs sa;
        if (batched) {
            const int64_t div = (l == L - 1) ? S.ratio : (1ll << (l + 1));
            int64_t* tl = d_targets + (size_t)l * (S.B + 1);
            SPC_LAUNCH(ctx, k_targets, grid_for(S.B, kThreads, maxb), kThreads, 0, S.B,
                       S.d_graph_ptr, div, tl);
            sa.B = S.B;
            sa.d_graph_ptr = cur_gptr;
            sa.d_targets = tl;
        } else {
            int64_t t = (l == L - 1) ? S.n_c : (g0.n >> (l + 1));
            if (t < S.n_c) t = S.n_c;
            if (t < 1) t = 1;
            sa.target = t;
        }
        SPC_TRY(run_score(ctx, cur, S.validate && l == 0, lv.score.p, S.schedule));
        lv.n = cur.n;
        lv.m = cur.m;
        int64_t n_c = 0;
        int32_t st = 0;
        SPC_TRY(run_select(ctx, cur, lv.score.p, sa, lv.lift.as<int32_t>(), nullptr, &n_c,
                           lv.graph_ptr_c.as<int64_t>(), &st));
        SPC_TRY(run_contract(ctx, cur, lv.lift.as<int32_t>(), n_c, lv));
        lv.mass_ptr = nullptr;
        if (S.self_mass) {
            // mass(U) = members' masses + this level's self-mass (the merged node of the proof
            // of Theorem 2 keeps the weight inside it)
            SPC_TRY(run_carry_mass(ctx, cur.n, lv.lift.as<int32_t>(), n_c, mass, lv.self_mass.p,
                                   cur.wtype, lv.mass, &lv.mass_ptr));
            mass = lv.mass_ptr;
        }
        lv.status = st;
        lv.wtype = cur.wtype;
        if (st == SPC_WARN_TARGET_NOT_REACHED) *warn = 1;
        ctx->n_levels = l + 1;
        GraphView nx;
        nx.n = n_c;
        nx.nnz = 2 * lv.m_c;
        nx.m = lv.m_c;
        nx.rowptr = lv.rowptr_c.as<int64_t>();
        nx.col = lv.col_c.as<int32_t>();
        nx.w = lv.w_c.p;
        nx.wtype = cur.wtype;
        // the next level scores G_c with each super-node's internal weight on its diagonal
        if (S.self_mass && l + 1 < L) {
            GraphView dg;
            SPC_TRY(run_diag_graph(ctx, nx, mass, dg));
            nx = dg;
        }
        SPC_CUDA(record_event(ctx, lv.ev1));
        cur = nx;
        cur_gptr = lv.graph_ptr_c.as<int64_t>();
    }
    // composed lift
    for (int l = 0; l < L;) {  // chains of up to kComposeMax lifts, continuing in place
        LiftChain ch{};
        ch.levels = 0;
        if (l > 0) ch.lift[ch.levels++] = lift_comp;
        while (l < L && ch.levels < kComposeMax)
            ch.lift[ch.levels++] = ctx->levels[l++].lift.as<int32_t>();
        SPC_LAUNCH(ctx, k_compose_all, grid_for(g0.n, kThreads, maxb), kThreads, 0, g0.n, ch,
                   lift_comp);
    }
    if (S.reorder) SPC_TRY(run_unpermute(ctx, g0.n, lift_comp, lift_total_dev));
    *n_c_final = cur.n;
    if (capturing(ctx)) return SPC_OK;
    SPC_TRY(sync_status(ctx));
    for (int l = 0; l < L; ++l) {
        float ms = -1.f;
        if (cudaEventElapsedTime(&ms, ctx->levels[l].ev0, ctx->levels[l].ev1) == cudaSuccess)
            ctx->levels[l].ms = ms;
        else
            (void)cudaGetLastError();
    }
    return SPC_OK;
}

// ---- recorded schedule, captured once, replayed ---------------------------------------------

__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

constexpr unsigned long long kPosMul = 0xD6E8FEB86659FD93ull;  // odd: positions stay distinct

// position-sensitive sum of mixed 8-byte words (4-byte words when the array is not 8-byte
// aligned or sized); four loads in flight per thread
__global__ void k_checksum(const void* __restrict__ p, int64_t bytes, unsigned long long salt,
                           unsigned long long* acc) {
    spc::pdl_wait();
    unsigned long long s = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (((uintptr_t)p & 7) == 0 && (bytes & 7) == 0) {
        const unsigned long long* w = static_cast<const unsigned long long*>(p);
        const int64_t words = bytes >> 3;
        int64_t i = t0;
        for (; i + 3 * stride < words; i += 4 * stride) {
            const unsigned long long a = w[i], b = w[i + stride], c = w[i + 2 * stride],
                                     d = w[i + 3 * stride];
            s += mix64(a ^ (kPosMul * (unsigned long long)i + salt));
            s += mix64(b ^ (kPosMul * (unsigned long long)(i + stride) + salt));
            s += mix64(c ^ (kPosMul * (unsigned long long)(i + 2 * stride) + salt));
            s += mix64(d ^ (kPosMul * (unsigned long long)(i + 3 * stride) + salt));
        }
        for (; i < words; i += stride) s += mix64(w[i] ^ (kPosMul * (unsigned long long)i + salt));
    } else {
        const uint32_t* w = static_cast<const uint32_t*>(p);
        for (int64_t i = t0; i < (bytes >> 2); i += stride)
            s += mix64((unsigned long long)w[i] ^ (kPosMul * (unsigned long long)i + salt + 1ull));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(acc, s);
}

static spc_status input_checksum(spc_context* ctx, const GraphView& v, const Schedule& S,
                                 unsigned long long* out) {
    Replay& R = ctx->replay;
    if (!R.d_hash) SPC_CUDA(cudaMalloc(&R.d_hash, 256));
    SPC_CUDA(cudaMemsetAsync(R.d_hash, 0, 8, ctx->stream));
    const int maxb = ctx->num_sms * 8;
    struct Arr { const void* p; int64_t bytes; unsigned long long salt; };
    const Arr arrs[4] = {{v.rowptr, (v.n + 1) * 8, 0x1111ull << 40},
                         {v.col, v.nnz * 4, 0x2222ull << 40},
                         {v.w, v.nnz * (int64_t)wsize(v.wtype), 0x3333ull << 40},
                         {S.d_graph_ptr, S.d_graph_ptr ? (S.B + 1) * 8 : 0, 0x4444ull << 40}};
    for (const Arr& ar : arrs) {
        if (!ar.p || ar.bytes <= 0) continue;
        SPC_LAUNCH(ctx, k_checksum, grid_for(ar.bytes / 32, kThreads, maxb), kThreads, 0, ar.p,
                   ar.bytes, ar.salt, R.d_hash);
    }
    SPC_CUDA(cudaMemcpyAsync(ctx->h_scalars + 24, R.d_hash, 8, cudaMemcpyDeviceToHost,
                             ctx->stream));
    SPC_CUDA(cudaStreamSynchronize(ctx->stream));
    *out = (unsigned long long)ctx->h_scalars[24];
    return SPC_OK;
}

static void drop_graph(Replay& R) {
    if (R.exec) cudaGraphExecDestroy(R.exec);
    if (R.graph) cudaGraphDestroy(R.graph);
    R.exec = nullptr;
    R.graph = nullptr;
}

static std::vector<int64_t> call_key(const GraphView& v, const Schedule& S) {
    return {(int64_t)(intptr_t)v.rowptr, (int64_t)(intptr_t)v.col, (int64_t)(intptr_t)v.w, v.n,
            v.nnz, (int64_t)v.wtype, S.levels, S.validate ? 1 : 0, S.schedule, S.n_c, S.B,
            (int64_t)(intptr_t)S.d_graph_ptr, S.ratio, S.self_mass ? 1 : 0,
            S.reorder ? 1 : 0};
}

static spc_status capture_graph(spc_context* ctx, const GraphView& v, const Schedule& S,
                                int32_t* lift_int) {
    Replay& R = ctx->replay;
    if (!R.cap_stream) SPC_CUDA(cudaStreamCreateWithFlags(&R.cap_stream, cudaStreamNonBlocking));
    if (!R.d_mismatch) SPC_CUDA(cudaMalloc(&R.d_mismatch, 256));
    for (auto& pr : R.timed) {
        ctx->timer.pool.push_back(pr.a);
        ctx->timer.pool.push_back(pr.b);
    }
    R.timed.clear();
    cudaStream_t user = ctx->stream;
    ctx->stream = R.cap_stream;
    R.mode = Replay::kCapture;
    R.pos = 0;
    const int64_t l0 = ctx->launches;
    cudaError_t e = cudaStreamBeginCapture(R.cap_stream, cudaStreamCaptureModeThreadLocal);
    spc_status st = SPC_ERR_CUDA;
    int64_t ncf = 0;
    int32_t warn = 0;
    if (e == cudaSuccess) st = run_levels(ctx, v, S, lift_int, &ncf, &warn);
    cudaGraph_t g = nullptr;
    if (e == cudaSuccess) e = cudaStreamEndCapture(R.cap_stream, &g);
    ctx->stream = user;
    R.mode = Replay::kDirect;
    const int64_t kernels = ctx->launches - l0;
    ctx->launches = l0;
    if (st != SPC_OK || e != cudaSuccess || R.pos != R.log.size() || g == nullptr) {
        (void)cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        return SPC_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&R.exec, g, 0);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        cudaGraphDestroy(g);
        R.exec = nullptr;
        return SPC_ERR_CUDA;
    }
    R.graph = g;
    R.graph_kernels = kernels;
    R.timer_substr = ctx->timer.on ? ctx->timer.substr : "";
    return SPC_OK;
}

// launch the captured schedule; > 0 return: the in-graph checks disagreed with the record
static spc_status replay_graph(spc_context* ctx, bool* mismatch) {
    Replay& R = ctx->replay;
    SPC_CUDA(cudaMemsetAsync(R.d_mismatch, 0, 4, ctx->stream));
    SPC_CUDA(cudaGraphLaunch(R.exec, ctx->stream));
    ctx->launches += R.graph_kernels;
    SPC_CUDA(cudaMemcpyAsync(ctx->h_scalars + 25, R.d_mismatch, 4, cudaMemcpyDeviceToHost,
                             ctx->stream));
    SPC_CUDA(cudaMemcpyAsync(ctx->h_status, ctx->d_status, 4, cudaMemcpyDeviceToHost,
                             ctx->stream));
    SPC_CUDA(cudaStreamSynchronize(ctx->stream));
    *mismatch = *reinterpret_cast<int32_t*>(ctx->h_scalars + 25) != 0;
    if (ctx->timer.on && ctx->timer.substr == R.timer_substr) {
        for (auto& pr : R.timed) {
            float ms = 0.f;
            SPC_CUDA(cudaEventElapsedTime(&ms, pr.a, pr.b));
            timer_add(ctx->timer, pr.name, ms, pr.bytes);
        }
    }
    return status_from_bits(*ctx->h_status);
}

// One coarsening call: replay the captured graph when this call repeats the recorded one on
// unchanged input, otherwise run host-driven (recording it when graphs are enabled).
static spc_status drive(spc_context* ctx, const GraphView& v, const Schedule& S, bool use_graph,
                        int64_t* ncf, int32_t* warn) {
    Replay& R = ctx->replay;
    ctx->replayed_last = 0;
    SPC_TRY(ensure(ctx, ctx->work.lift_final, ((size_t)v.n + 1) * 4));
    int32_t* lift_int = ctx->work.lift_final.as<int32_t>();
    const std::vector<int64_t> key = call_key(v, S);
    const std::string tsub = ctx->timer.on ? ctx->timer.substr : "";
    unsigned long long hsh = 0;
    if (use_graph) SPC_TRY(input_checksum(ctx, v, S, &hsh));
    if (use_graph && R.recorded && R.key == key && R.hash == hsh) {
        if (R.exec && R.timer_substr != tsub) drop_graph(R);
        if (!R.exec && capture_graph(ctx, v, S, lift_int) != SPC_OK) {
            drop_graph(R);
            R.recorded = false;
        }
        if (R.exec) {
            bool mismatch = false;
            const spc_status st = replay_graph(ctx, &mismatch);
            if (st < 0) return st;
            if (!mismatch) {
                ctx->replayed_last = 1;
                const int L = (int)R.metas.size();
                for (int l = 0; l < L; ++l) {
                    LevelBufs& lv = ctx->levels[l];
                    lv.n = R.metas[l].n; lv.m = R.metas[l].m; lv.n_c = R.metas[l].n_c;
                    lv.m_c = R.metas[l].m_c; lv.m_inter = R.metas[l].m_inter;
                    lv.status = R.metas[l].status; lv.wtype = R.metas[l].wtype;
                    lv.mass_ptr = R.metas[l].mass_ptr;
                    float ms = -1.f;
                    if (cudaEventElapsedTime(&ms, lv.ev0, lv.ev1) != cudaSuccess) {
                        (void)cudaGetLastError();
                        ms = -1.f;
                    }
                    lv.ms = ms;
                }
                ctx->n_levels = L;
                *ncf = R.n_c_final;
                *warn = R.warn;
                return SPC_OK;
            }
            drop_graph(R);  // the device disagreed with the record: run host-driven again
            R.recorded = false;
        }
    }
    R.mode = use_graph ? Replay::kRecord : Replay::kDirect;
    R.log.clear();
    const spc_status st = run_levels(ctx, v, S, lift_int, ncf, warn);
    R.mode = Replay::kDirect;
    drop_graph(R);
    R.recorded = false;
    if (st == SPC_OK && use_graph) {
        R.recorded = true;
        R.key = key;
        R.hash = hsh;
        R.metas.clear();
        for (int l = 0; l < ctx->n_levels; ++l) {
            const LevelBufs& lv = ctx->levels[l];
            LevelMeta mt;
            mt.n = lv.n; mt.m = lv.m; mt.n_c = lv.n_c; mt.m_c = lv.m_c; mt.m_inter = lv.m_inter;
            mt.status = lv.status; mt.wtype = lv.wtype;
            mt.mass_ptr = lv.mass_ptr;
            R.metas.push_back(mt);
        }
        R.n_c_final = *ncf;
        R.warn = *warn;
    }
    return st;
}

}  // namespace spc

using namespace spc;

// ============================================================================================
extern "C" {

const char* spc_status_string(spc_status s) {
    switch (s) {
        case SPC_OK: return "SPC_OK";
        case SPC_WARN_TARGET_NOT_REACHED: return "SPC_WARN_TARGET_NOT_REACHED";
        case SPC_ERR_INVALID_ARG: return "SPC_ERR_INVALID_ARG";
        case SPC_ERR_NOT_SYMMETRIC: return "SPC_ERR_NOT_SYMMETRIC";
        case SPC_ERR_SELF_LOOP: return "SPC_ERR_SELF_LOOP";
        case SPC_ERR_UNSORTED: return "SPC_ERR_UNSORTED";
        case SPC_ERR_OOM: return "SPC_ERR_OOM";
        case SPC_ERR_CUDA: return "SPC_ERR_CUDA";
        case SPC_ERR_TIMEOUT: return "SPC_ERR_TIMEOUT";
        case SPC_ERR_OVERFLOW: return "SPC_ERR_OVERFLOW";
        case SPC_ERR_BAD_WEIGHT: return "SPC_ERR_BAD_WEIGHT";
        case SPC_ERR_TOO_LARGE: return "SPC_ERR_TOO_LARGE";
    }
    return "SPC_UNKNOWN_STATUS";
}

spc_options spc_default_options(void) {
    spc_options o;
    o.levels = 1;
    o.validate = 1;
    o.use_graph = 1;
    o.schedule = 0;
    o.self_mass = 1;
    o.reorder = 0;
    return o;
}

spc_status spc_context_create(spc_context** out, const spc_allocator* allocator, void* stream) {
    if (!out) return SPC_ERR_INVALID_ARG;
    *out = nullptr;
    spc_context* ctx = new (std::nothrow) spc_context();
    if (!ctx) return SPC_ERR_OOM;
    ctx->stream = static_cast<cudaStream_t>(stream);
    if (allocator && allocator->alloc && allocator->free) {
        ctx->allocator = *allocator;
        ctx->has_allocator = true;
    }
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, 256);
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_status, 256);
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_scalars, 256);
    if (e != cudaSuccess) {
        set_last_cuda_error(e, "spc_context_create", __FILE__, __LINE__);
        if (ctx->d_status) cudaFree(ctx->d_status);
        if (ctx->h_status) cudaFreeHost(ctx->h_status);
        delete ctx;
        return SPC_ERR_CUDA;
    }
    cudaMemset(ctx->d_status, 0, 256);
    {
        std::random_device rd;  // the symmetry fingerprint's key, unknown to whoever built the input
        for (auto& k : ctx->sym_key) k = ((uint64_t)rd() << 32) ^ (uint64_t)rd();
    }
    *out = ctx;
    return SPC_OK;
}

void spc_context_destroy(spc_context* ctx) {
    if (!ctx) return;
    free_all(ctx);
    for (auto& lv : ctx->levels) {
        if (lv.ev0) cudaEventDestroy(lv.ev0);
        if (lv.ev1) cudaEventDestroy(lv.ev1);
    }
    for (auto& pr : ctx->timer.pending) {
        cudaEventDestroy(pr.a);
        cudaEventDestroy(pr.b);
    }
    for (auto ev : ctx->timer.pool) cudaEventDestroy(ev);
    for (auto& pr : ctx->replay.timed) {
        cudaEventDestroy(pr.a);
        cudaEventDestroy(pr.b);
    }
    drop_graph(ctx->replay);
    if (ctx->replay.d_mismatch) cudaFree(ctx->replay.d_mismatch);
    if (ctx->replay.d_hash) cudaFree(ctx->replay.d_hash);
    if (ctx->d_ops) cudaFree(ctx->d_ops);
    if (ctx->replay.cap_stream) cudaStreamDestroy(ctx->replay.cap_stream);
    if (ctx->side_stream) cudaStreamDestroy(ctx->side_stream);
    for (auto ev : ctx->branch_ev)
        if (ev) cudaEventDestroy(ev);
    for (auto ev : ctx->tune_ev)
        if (ev) cudaEventDestroy(ev);
    cudaFree(ctx->d_status);
    cudaFreeHost(ctx->h_status);
    cudaFreeHost(ctx->h_scalars);
    delete ctx;
}

spc_status spc_context_set_wait_limit(spc_context* ctx, uint32_t iterations) {
    if (!ctx) return SPC_ERR_INVALID_ARG;
    SPC_CUDA(cudaSetDevice(ctx->device));
    SPC_CUDA(cudaMemcpyAsync(ctx->d_status + 1, &iterations, sizeof(uint32_t),
                             cudaMemcpyHostToDevice, ctx->stream));
    SPC_CUDA(cudaStreamSynchronize(ctx->stream));
    return SPC_OK;
}

spc_status spc_context_set_stream(spc_context* ctx, void* stream) {
    if (!ctx) return SPC_ERR_INVALID_ARG;
    SPC_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->stream = static_cast<cudaStream_t>(stream);
    return SPC_OK;
}

spc_status spc_copy(spc_context* ctx, void* dst, const void* src, size_t bytes) {
    if (!ctx || (bytes && (!dst || !src))) return SPC_ERR_INVALID_ARG;
    SPC_TRY(copy_out(ctx, dst, src, bytes));
    SPC_CUDA(cudaStreamSynchronize(ctx->stream));
    return SPC_OK;
}

spc_status spc_score(spc_context* ctx, const spc_csr* g, void* f_out, int64_t* m_out) {
    SPC_TRY(begin_call(ctx));
    SPC_TRY(check_csr(g));
    if (!f_out) return SPC_ERR_INVALID_ARG;
    GraphView v;
    SPC_TRY(stage_graph(ctx, g, v));
    SPC_TRY(reserve_work(ctx, v.n, v.nnz / 2, 1));
    const size_t fsz = score_is_f32(v.wtype) ? 4 : 8;
    const bool dev_out = is_device_ptr(f_out);
    Buf& tmp = ctx->work.sel_key;  // sized >= m * 8
    SPC_TRY(run_score(ctx, v, true, dev_out ? f_out : tmp.p, 1));
    if (!dev_out) SPC_TRY(copy_out(ctx, f_out, tmp.p, (size_t)v.m * fsz));
    if (m_out) *m_out = v.m;
    return sync_status(ctx);
}

spc_status spc_sort_fitness(spc_context* ctx, int64_t m, const void* f, spc_dtype ftype,
                            int32_t* order_out) {
    SPC_TRY(begin_call(ctx));
    if (m < 0 || (m > 0 && (!f || !order_out))) return SPC_ERR_INVALID_ARG;
    if (ftype != SPC_F32 && ftype != SPC_F64) return SPC_ERR_INVALID_ARG;
    if (m >= INT32_MAX) return SPC_ERR_TOO_LARGE;
    SPC_TRY(reserve_work(ctx, 1, m, 1));
    const size_t fsz = ftype == SPC_F32 ? 4 : 8;
    const void* fd;
    SPC_TRY(stage_in(ctx, f, (size_t)m * fsz, ctx->work.stage_w, &fd));
    const bool dev_out = is_device_ptr(order_out);
    int32_t* ord = dev_out ? order_out : ctx->work.c_val.as<int32_t>();
    SPC_TRY(run_sort_fitness(ctx, m, fd, ftype == SPC_F32, ord));
    if (!dev_out) SPC_TRY(copy_out(ctx, order_out, ord, (size_t)m * 4));
    return sync_status(ctx);
}

spc_status spc_select_merges(spc_context* ctx, const spc_csr* g, const void* f, int64_t n_c,
                             int32_t* lift_out, uint8_t* merged_out, int64_t* n_c_actual) {
    SPC_TRY(begin_call(ctx));
    SPC_TRY(check_csr(g));
    if (!f || !lift_out || n_c < 1) return SPC_ERR_INVALID_ARG;
    GraphView v;
    SPC_TRY(stage_graph(ctx, g, v));
    SPC_TRY(reserve_work(ctx, v.n, v.nnz / 2, 1));
    if (ctx->levels.empty()) ctx->levels.resize(1);
    SPC_TRY(reserve_level(ctx, ctx->levels[0], v.n, v.nnz / 2, 1));
    SPC_TRY(run_score(ctx, v, true, nullptr, 1));  // edge list only
    const size_t fsz = score_is_f32(v.wtype) ? 4 : 8;
    const void* fd;
    SPC_TRY(stage_in(ctx, f, (size_t)v.m * fsz, ctx->levels[0].score, &fd));
    SelectArgs sa;
    sa.target = n_c;
    const bool dev_lift = is_device_ptr(lift_out);
    const bool dev_merged = merged_out && is_device_ptr(merged_out);
    int32_t* lift = dev_lift ? lift_out : ctx->levels[0].lift.as<int32_t>();
    uint8_t* merged = merged_out ? (dev_merged ? merged_out : ctx->work.c_flag.as<uint8_t>()) : nullptr;
    int64_t nc = 0;
    int32_t st = 0;
    SPC_TRY(run_select(ctx, v, fd, sa, lift, merged, &nc, nullptr, &st));
    if (!dev_lift) SPC_TRY(copy_out(ctx, lift_out, lift, (size_t)v.n * 4));
    if (merged_out && !dev_merged) SPC_TRY(copy_out(ctx, merged_out, merged, (size_t)v.m));
    if (n_c_actual) *n_c_actual = nc;
    SPC_TRY(sync_status(ctx));
    return (spc_status)st;
}

spc_status spc_contract(spc_context* ctx, const spc_csr* g, const int32_t* lift, int64_t n_c,
                        int64_t* m_c_out) {
    SPC_TRY(begin_call(ctx));
    SPC_TRY(check_csr(g));
    if (!lift || n_c < 1 || n_c > (g->n > 0 ? g->n : 1)) return SPC_ERR_INVALID_ARG;
    GraphView v;
    SPC_TRY(stage_graph(ctx, g, v));
    SPC_TRY(reserve_work(ctx, v.n, v.nnz / 2, 1));
    if (ctx->levels.empty()) ctx->levels.resize(1);
    LevelBufs& lv = ctx->levels[0];
    SPC_TRY(reserve_level(ctx, lv, v.n, v.nnz / 2, 1));
    SPC_TRY(run_score(ctx, v, true, nullptr, 1));
    const void* ld;
    SPC_TRY(stage_in(ctx, lift, (size_t)v.n * 4, ctx->work.stage_lift, &ld));
    SPC_CUDA(cudaMemcpyAsync(lv.lift.p, ld, (size_t)v.n * 4, cudaMemcpyDeviceToDevice,
                             ctx->stream));
    if (v.n > 0) {
        SPC_LAUNCH(ctx, k_check_lift, grid_for(v.n, kThreads, ctx->num_sms * 8), kThreads, 0,
                   v.n, lv.lift.as<int32_t>(), n_c, ctx->d_status);
    }
    SPC_TRY(sync_status(ctx));  // an out-of-range id must not reach the contraction
    ctx->has_result = false;
    ctx->reorder_n = 0;
    SPC_TRY(run_contract(ctx, v, lv.lift.as<int32_t>(), n_c, lv));
    lv.n = v.n;
    lv.m = v.m;
    lv.status = SPC_OK;
    lv.wtype = v.wtype;
    lv.ms = -1.f;
    lv.mass_ptr = nullptr;
    ctx->n_levels = 1;
    if (m_c_out) *m_c_out = lv.m_c;
    return sync_status(ctx);
}

spc_status spc_coarsen(spc_context* ctx, const spc_csr* g, int64_t n_c, const spc_options* options,
                       int32_t* lift_out, int64_t* n_c_actual) {
    SPC_TRY(begin_call(ctx));
    SPC_TRY(check_csr(g));
    if (!lift_out || n_c < 1) return SPC_ERR_INVALID_ARG;
    spc_options o = options ? *options : spc_default_options();
    GraphView v;
    SPC_TRY(stage_graph(ctx, g, v));
    Schedule S;
    S.levels = o.levels < 1 ? 1 : o.levels;
    S.validate = o.validate != 0;
    S.schedule = o.schedule;
    S.self_mass = o.self_mass != 0;
    S.reorder = o.reorder != 0;
    S.n_c = n_c;
    int64_t ncf = 0;
    int32_t warn = 0;
    ctx->has_result = false;
    ctx->reorder_n = 0;
    SPC_TRY(drive(ctx, v, S, o.use_graph != 0, &ncf, &warn));
    ctx->has_result = true;
    ctx->reorder_n = S.reorder ? v.n : 0;
    SPC_TRY(copy_out(ctx, lift_out, ctx->work.lift_final.p, (size_t)v.n * 4));
    SPC_CUDA(cudaStreamSynchronize(ctx->stream));
    if (n_c_actual) *n_c_actual = ncf;
    return warn ? SPC_WARN_TARGET_NOT_REACHED : SPC_OK;
}

spc_status spc_coarsen_batched(spc_context* ctx, const spc_csr* g, const int64_t* graph_ptr,
                               int64_t B, int64_t ratio, const spc_options* options,
                               int32_t* lift_out, int64_t* graph_ptr_c_out) {
    SPC_TRY(begin_call(ctx));
    SPC_TRY(check_csr(g));
    if (!graph_ptr || B < 1 || ratio < 1 || !lift_out) return SPC_ERR_INVALID_ARG;
    spc_options o = options ? *options : spc_default_options();
    const int L = o.levels < 1 ? 1 : o.levels;
    if (L > 1 && (1ll << L) != ratio) return SPC_ERR_INVALID_ARG;
    GraphView v;
    SPC_TRY(stage_graph(ctx, g, v));
    const void* gp;
    SPC_TRY(ensure(ctx, ctx->work.stage_gptr, ((size_t)B + 1) * 8 * (L + 2)));
    // level-0 graph_ptr lives in the last slot of stage_gptr (targets use the first L slots)
    int64_t* gp_dev = ctx->work.stage_gptr.as<int64_t>() + (size_t)(L + 1) * (B + 1);
    SPC_TRY(stage_in(ctx, graph_ptr, ((size_t)B + 1) * 8, ctx->work.seg_start, &gp));
    SPC_CUDA(cudaMemcpyAsync(gp_dev, gp, ((size_t)B + 1) * 8, cudaMemcpyDeviceToDevice,
                             ctx->stream));
    Schedule S;
    S.levels = L;
    S.validate = o.validate != 0;
    S.schedule = o.schedule;
    S.self_mass = o.self_mass != 0;
    S.B = B;
    S.d_graph_ptr = gp_dev;
    S.ratio = ratio;
    int64_t ncf = 0;
    int32_t warn = 0;
    ctx->has_result = false;
    ctx->reorder_n = 0;
    SPC_TRY(drive(ctx, v, S, o.use_graph != 0, &ncf, &warn));
    ctx->has_result = true;
    SPC_TRY(copy_out(ctx, lift_out, ctx->work.lift_final.p, (size_t)v.n * 4));
    if (graph_ptr_c_out)
        SPC_TRY(copy_out(ctx, graph_ptr_c_out, ctx->levels[L - 1].graph_ptr_c.p,
                         ((size_t)B + 1) * 8));
    SPC_CUDA(cudaStreamSynchronize(ctx->stream));
    return warn ? SPC_WARN_TARGET_NOT_REACHED : SPC_OK;
}

void spc_result_free(spc_context* ctx, spc_result* r) {
    if (!ctx || !r) return;
    cudaStreamSynchronize(ctx->stream);
    void* ps[6] = {r->lift, r->emap, r->rowptr_c, r->col_c, r->w_c, r->mass};
    for (void* p : ps) free_owned(ctx, p);
    *r = spc_result{};
}

spc_status spc_take_result(spc_context* ctx, spc_result* out) {
    SPC_TRY(begin_call(ctx));
    if (!out) return SPC_ERR_INVALID_ARG;
    *out = spc_result{};
    if (!ctx->has_result || ctx->n_levels < 1) return SPC_ERR_INVALID_ARG;
    const LevelBufs& l0 = ctx->levels[0];
    const LevelBufs& lz = ctx->levels[ctx->n_levels - 1];
    spc_result r{};
    r.n = l0.n;
    r.m = l0.m;
    r.n_c = lz.n_c;
    r.m_c = lz.m_c;
    r.wtype = lz.wtype;
    const size_t ws = wsize(r.wtype), acc = accsize(r.wtype);
    r.lift = static_cast<int32_t*>(alloc_owned(ctx, (size_t)r.n * 4));
    r.emap = static_cast<int32_t*>(alloc_owned(ctx, (size_t)r.m * 4));
    r.rowptr_c = static_cast<int64_t*>(alloc_owned(ctx, (size_t)(r.n_c + 1) * 8));
    r.col_c = static_cast<int32_t*>(alloc_owned(ctx, (size_t)r.m_c * 2 * 4));
    r.w_c = alloc_owned(ctx, (size_t)r.m_c * 2 * ws);
    if (lz.mass_ptr) r.mass = alloc_owned(ctx, (size_t)r.n_c * acc);
    if (!r.lift || !r.emap || !r.rowptr_c || !r.col_c || !r.w_c || (lz.mass_ptr && !r.mass)) {
        spc_result_free(ctx, &r);
        return SPC_ERR_OOM;
    }
    spc_status st = SPC_OK;
    auto cp = [&](void* dst, const void* src, size_t bytes) {
        if (st == SPC_OK && bytes &&
            cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
            st = SPC_ERR_CUDA;
    };
    cp(r.lift, ctx->work.lift_final.p, (size_t)r.n * 4);
    cp(r.emap, l0.emap.p, (size_t)r.m * 4);
    cp(r.rowptr_c, lz.rowptr_c.p, (size_t)(r.n_c + 1) * 8);
    cp(r.col_c, lz.col_c.p, (size_t)r.m_c * 2 * 4);
    cp(r.w_c, lz.w_c.p, (size_t)r.m_c * 2 * ws);
    if (r.mass) cp(r.mass, lz.mass_ptr, (size_t)r.n_c * acc);
    for (int l = 1; l < ctx->n_levels && st == SPC_OK && r.m > 0; ++l) {
        st = [&]() -> spc_status {
            SPC_LAUNCH(ctx, k_compose_emap, grid_for(r.m, kThreads, ctx->num_sms * 8), kThreads, 0,
                       r.m, ctx->levels[l].emap.as<int32_t>(), r.emap);
            return SPC_OK;
        }();
    }
    if (st == SPC_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) st = SPC_ERR_CUDA;
    if (st != SPC_OK) {
        (void)cudaGetLastError();
        spc_result_free(ctx, &r);
        return st;
    }
    *out = r;
    return SPC_OK;
}

spc_status spc_get_reorder(spc_context* ctx, int32_t* perm_out) {
    SPC_TRY(begin_call(ctx));
    if (!perm_out || ctx->reorder_n <= 0) return SPC_ERR_INVALID_ARG;
    SPC_TRY(copy_out(ctx, perm_out, ctx->work.ro_perm.p, (size_t)ctx->reorder_n * 4));
    SPC_CUDA(cudaStreamSynchronize(ctx->stream));
    return SPC_OK;
}

int32_t spc_level_count(const spc_context* ctx) { return ctx ? ctx->n_levels : 0; }

spc_status spc_get_level(const spc_context* ctx, int32_t level, spc_level* out) {
    if (!ctx || !out || level < 0 || level >= ctx->n_levels) return SPC_ERR_INVALID_ARG;
    const LevelBufs& lv = ctx->levels[level];
    out->n = lv.n;
    out->m = lv.m;
    out->n_c = lv.n_c;
    out->m_c = lv.m_c;
    out->m_inter = lv.m_inter;
    out->status = lv.status;
    out->wtype = lv.wtype;
    out->score = lv.score.p;
    out->scoretype = lv.wtype == SPC_F32 ? SPC_F32 : SPC_F64;
    out->lift = lv.lift.as<int32_t>();
    out->emap = lv.emap.as<int32_t>();
    out->self_mass = lv.self_mass.p;
    out->a_und = lv.a_und.p;
    out->rowptr_c = lv.rowptr_c.as<int64_t>();
    out->col_c = lv.col_c.as<int32_t>();
    out->w_c = lv.w_c.p;
    out->perm = lv.perm.as<int32_t>();
    out->seg = lv.seg.as<int32_t>();
    out->graph_ptr_c = lv.graph_ptr_c.as<int64_t>();
    out->ms = lv.ms;
    out->mass = lv.mass_ptr;
    return SPC_OK;
}

spc_status spc_contract_forward(spc_context* ctx, const int32_t* perm, const int32_t* seg,
                                int64_t m_c, const void* w_und, spc_dtype wtype, void* a_und) {
    SPC_TRY(begin_call(ctx));
    if (m_c < 0 || (m_c > 0 && (!perm || !seg || !w_und || !a_und))) return SPC_ERR_INVALID_ARG;
    SPC_TRY(run_contract_forward(ctx, perm, seg, m_c, w_und, wtype, a_und));
    return sync_status(ctx);
}

spc_status spc_contract_backward(spc_context* ctx, const int32_t* emap, int64_t m,
                                 const void* grad_a, void* grad_w, spc_dtype dtype) {
    SPC_TRY(begin_call(ctx));
    if (m < 0 || (m > 0 && (!emap || !grad_a || !grad_w))) return SPC_ERR_INVALID_ARG;
    SPC_TRY(run_contract_backward(ctx, emap, m, grad_a, grad_w, dtype));
    return sync_status(ctx);
}

spc_status spc_pool_features(spc_context* ctx, int64_t n, const int32_t* lift, int64_t n_c,
                             int64_t F, spc_dtype dtype, const void* x, void* xc_out) {
    SPC_TRY(begin_call(ctx));
    if (n < 0 || n_c < 1 || F < 1 || n_c > INT32_MAX || n >= (int64_t)INT32_MAX ||
        (dtype != SPC_F32 && dtype != SPC_F64) || (n > 0 && (!lift || !x)) || !xc_out)
        return SPC_ERR_INVALID_ARG;
    if (n > (int64_t(1) << 62) / F || n_c > (int64_t(1) << 62) / F) return SPC_ERR_TOO_LARGE;
    SPC_TRY(run_pool_forward(ctx, n, lift, n_c, F, dtype, x, xc_out));
    return sync_status(ctx);
}

spc_status spc_pool_features_backward(spc_context* ctx, int64_t n, const int32_t* lift,
                                      int64_t n_c, int64_t F, spc_dtype dtype,
                                      const void* grad_xc, void* grad_x_out) {
    SPC_TRY(begin_call(ctx));
    if (n < 0 || n_c < 1 || F < 1 || n_c > INT32_MAX || n >= (int64_t)INT32_MAX ||
        (dtype != SPC_F32 && dtype != SPC_F64) || (n > 0 && (!lift || !grad_x_out)) || !grad_xc)
        return SPC_ERR_INVALID_ARG;
    if (n > (int64_t(1) << 62) / F || n_c > (int64_t(1) << 62) / F) return SPC_ERR_TOO_LARGE;
    SPC_TRY(run_pool_backward(ctx, n, lift, n_c, F, dtype, grad_xc, grad_x_out));
    return sync_status(ctx);
}

spc_status spc_compose_emap(spc_context* ctx, int32_t* emap_out) {
    SPC_TRY(begin_call(ctx));
    if (!emap_out || ctx->n_levels < 1) return SPC_ERR_INVALID_ARG;
    const int64_t m = ctx->levels[0].m;
    const bool dev = is_device_ptr(emap_out);
    int32_t* em = dev ? emap_out : ctx->work.c_val.as<int32_t>();
    SPC_CUDA(cudaMemcpyAsync(em, ctx->levels[0].emap.p, (size_t)m * 4, cudaMemcpyDeviceToDevice,
                             ctx->stream));
    for (int l = 1; l < ctx->n_levels; ++l) {
        SPC_LAUNCH(ctx, k_compose_emap, grid_for(m, kThreads, ctx->num_sms * 8), kThreads, 0, m,
                   ctx->levels[l].emap.as<int32_t>(), em);
    }
    if (!dev) SPC_TRY(copy_out(ctx, emap_out, em, (size_t)m * 4));
    return sync_status(ctx);
}

spc_status spc_time_kernel(spc_context* ctx, const char* kernel_substr) {
    if (!ctx) return SPC_ERR_INVALID_ARG;
    Timer& t = ctx->timer;
    SPC_CUDA(cudaStreamSynchronize(ctx->stream));
    for (auto& pr : t.pending) {
        t.pool.push_back(pr.a);
        t.pool.push_back(pr.b);
    }
    t.pending.clear();
    t.per_kernel.clear();
    t.launches = 0;
    t.total_ms = 0.0;
    t.on = kernel_substr && kernel_substr[0];
    t.substr = t.on ? kernel_substr : "";
    if (t.on) {
        if (!ctx->d_ops) SPC_CUDA(cudaMalloc(&ctx->d_ops, 6 * sizeof(unsigned long long)));
        SPC_CUDA(cudaMemset(ctx->d_ops, 0, 6 * sizeof(unsigned long long)));
    }
    return SPC_OK;
}

static spc_status drain_timer(spc_context* ctx) {
    Timer& t = ctx->timer;
    SPC_CUDA(cudaStreamSynchronize(ctx->stream));
    for (auto& pr : t.pending) {
        float ms = 0.f;
        SPC_CUDA(cudaEventElapsedTime(&ms, pr.a, pr.b));
        timer_add(t, pr.name, ms, pr.bytes);
        t.pool.push_back(pr.a);
        t.pool.push_back(pr.b);
    }
    t.pending.clear();
    return SPC_OK;
}

spc_status spc_kernel_time(spc_context* ctx, int64_t* launches, double* total_ms) {
    if (!ctx) return SPC_ERR_INVALID_ARG;
    SPC_TRY(drain_timer(ctx));
    if (launches) *launches = ctx->timer.launches;
    if (total_ms) *total_ms = ctx->timer.total_ms;
    return SPC_OK;
}

spc_status spc_kernel_profile(spc_context* ctx, char* buf, size_t len) {
    if (!ctx || (!buf && len)) return SPC_ERR_INVALID_ARG;
    SPC_TRY(drain_timer(ctx));
    unsigned long long ops[6] = {0, 0, 0, 0, 0, 0};
    if (ctx->d_ops) SPC_CUDA(cudaMemcpy(ops, ctx->d_ops, sizeof(ops), cudaMemcpyDeviceToHost));
    std::string out;
    char line[512];
    for (auto& pk : ctx->timer.per_kernel) {
        unsigned long long fp = 0;
        if (pk.name.find("k_score_edges") != std::string::npos) fp = ops[0] + ops[1];
        if (pk.name.find("k_score_warp_row") != std::string::npos) fp = ops[2] + ops[3];
        if (pk.name.find("k_score_staged") != std::string::npos) fp = ops[4] + ops[5];
        snprintf(line, sizeof(line), "%s\t%lld\t%.6f\t%.0f\t%llu\n", pk.name.c_str(),
                 (long long)pk.launches, pk.ms, pk.bytes, fp);
        out += line;
    }
    if (len) {
        size_t k = out.size() < len - 1 ? out.size() : len - 1;
        memcpy(buf, out.data(), k);
        buf[k] = 0;
    }
    return out.size() < len ? SPC_OK : SPC_ERR_INVALID_ARG;
}

int64_t spc_launch_count(const spc_context* ctx) { return ctx ? ctx->launches : 0; }

int spc_last_call_replayed(const spc_context* ctx) { return ctx ? ctx->replayed_last : 0; }

}  // extern "C"
