/*
 * spcoarsen -- GB300 (sm_103a) spectral-bound graph coarsening.
 *
 * C ABI of libspcoarsen.so.  It implements the data-parallel path of Brissette, Huang and
 * Slota, "Parallel coarsening of graph data with spectral guarantees" (arXiv 2204.11757):
 *   1. every undirected edge (a, b) gets the score f(a, b) = || w_a/d_a - w_b/d_b ||_1
 *      (Theorem 1, Algorithm 1 fitness loop);
 *   2. edges are taken in ascending (f, edge id) order and their end points merged into
 *      super-nodes, passing over pairs already merged, until n_c super-nodes remain
 *      (Algorithm 1 sort and merge loop);
 *   3. the graph is contracted: a(U, V) = sum of w(x, y) over x in U, y in V (Definition 1),
 *      and the step is repeated level by level on the coarse graph (Section 4, recomputing the
 *      norms after partial coarsening).
 *
 * Conventions shared by every entry point
 *   - Graphs are symmetric CSR: rowptr int64[n+1] (rowptr[0] = 0, rowptr[n] = nnz = 2m),
 *     col int32[nnz] strictly ascending inside each row, no self-loops, every entry (x, y, w)
 *     mirrored by (y, x, w) with a bit-identical weight, weights finite and > 0.
 *   - The undirected edge id (eid) of {u, v}, u < v, is its rank in lexicographic (u, v)
 *     order, i.e. the order of the upper-triangle entries read row by row.  m < 2^31.
 *   - Weight types: SPC_I32 (degrees and scores exact in int64/binary64; coarse sums must fit
 *     in int32), SPC_F32 (degrees, normalised rows and scores in binary32), SPC_F64 (binary64).
 *     Scores are binary64 for SPC_I32/SPC_F64 and binary32 for SPC_F32.  All arithmetic is
 *     IEEE round-to-nearest without FMA contraction, in a fixed order (sums run in ascending
 *     column / edge id), so results are reproducible bit for bit.
 *   - Pointers: unless stated otherwise a pointer may be device memory or host memory (pinned
 *     or pageable); the library classifies it with cudaPointerGetAttributes and stages host
 *     data through its own device workspace.  Inputs are only read.  All work is issued on the
 *     context's stream; an entry point returns after that stream has finished the call's work
 *     (it synchronises once, to read the status word and data-dependent sizes).
 *   - Errors: every entry point returns an spc_status and never aborts the process.  Invalid
 *     input detected on the device is reported through a device status word read back at the
 *     end of the call.  Device-side waits are bounded; a wait that gives up reports
 *     SPC_ERR_TIMEOUT.  After an error the outputs are unspecified but the context stays usable.
 *   - Threading: a context is not thread-safe; use one context per host thread / stream.
 */
#ifndef SPCOARSEN_H
#define SPCOARSEN_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SPC_API __attribute__((visibility("default")))
#else
#define SPC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPC_OK = 0,
    SPC_WARN_TARGET_NOT_REACHED = 1, /* fewer merges possible than asked (more components than
                                        n_c); the partition is the connected components      */
    SPC_ERR_INVALID_ARG = -1,        /* null pointer, n_c < 1, bad dtype, sizes inconsistent  */
    SPC_ERR_NOT_SYMMETRIC = -2,      /* an entry (x,y,w) without a bit-identical (y,x,w)       */
    SPC_ERR_SELF_LOOP = -3,          /* an entry (x,x)                                         */
    SPC_ERR_UNSORTED = -4,           /* columns not strictly ascending, or out of [0,n), or a
                                        rowptr that is not monotone                            */
    SPC_ERR_OOM = -5,                /* workspace allocation failed                            */
    SPC_ERR_CUDA = -6,               /* a CUDA runtime call failed                             */
    SPC_ERR_TIMEOUT = -7,            /* a bounded device-side wait gave up                     */
    SPC_ERR_OVERFLOW = -8,           /* an SPC_I32 coarse weight does not fit in int32         */
    SPC_ERR_BAD_WEIGHT = -9,         /* a weight <= 0, NaN or infinite                         */
    SPC_ERR_TOO_LARGE = -10          /* an input exceeds a fixed size limit of the entry point:
                                        m >= 2^31 or n >= 2^31 everywhere, and the smaller
                                        limit stated at an entry point's declaration          */
} spc_status;

typedef enum { SPC_I32 = 0, SPC_F32 = 1, SPC_F64 = 2 } spc_dtype;

/* A symmetric CSR graph (see the conventions above). */
typedef struct {
    int64_t n;              /* number of nodes                                   */
    int64_t nnz;            /* stored entries, 2m                                */
    const int64_t* rowptr;  /* [n+1]                                             */
    const int32_t* col;     /* [nnz]                                             */
    const void* w;          /* [nnz] of type wtype                               */
    spc_dtype wtype;
} spc_csr;

/* Device-memory allocator used for the context's workspace (for example PyTorch's caching
 * allocator).  alloc returns a device pointer aligned to at least 256 bytes, or NULL.  When
 * the allocator passed to spc_context_create is NULL the library uses cudaMalloc/cudaFree. */
typedef struct {
    void* (*alloc)(void* ctx, size_t bytes);
    void (*free)(void* ctx, void* ptr);
    void* ctx;
} spc_allocator;

typedef struct {
    int32_t levels;     /* 0 or 1: one pass of Algorithm 1 straight to n_c.  L > 1: L levels,
                           level l (1-based) targets max(n_c, floor(n / 2^l)) super-nodes and
                           the last level targets n_c (Section 4: recompute the norms after
                           partial coarsening; Section 3 coarsens by halves).                 */
    int32_t validate;   /* 1: check the input graph (S0) before the first level; 0: trust it.
                           Rows (order, range, self-loops, weights) are checked exactly, and so
                           is symmetry for int32 and binary64 weights; for binary32 weights
                           symmetry is checked by a keyed 64-bit fingerprint of all entries
                           (an asymmetric graph passes with probability about 2^-64) */
    int32_t use_graph;  /* 1: capture the schedule in a CUDA graph and replay it on later calls
                           with the same shapes; 0: launch kernel by kernel                   */
    int32_t schedule;   /* score-kernel schedule: 0 auto (autotuned), 1 edge tiles
                           (one thread per edge), 2 warp per row, 3 staged rows (a warp
                           moves the rows of 32 edges into shared memory, then one thread
                           per edge); every schedule gives the same bits                    */
    int32_t self_mass;  /* multilevel reading (levels > 1 only; the first level is the same
                           either way).  1 (default): a super-node keeps the weight inside it.
                           Each level after the first scores its input graph with the diagonal
                           entry (U, U) = 2 mass(U) of every super-node U with internal weight,
                           stored in its ascending-column place, so it counts in U's degree and
                           in the scores of U's edges.  mass(U) is U's accumulated internal
                           weight: the masses of its members (ascending member id, summed left
                           to right from 0) plus this level's self-mass of U.  This is the merged
                           node (w_a + w_b) / (d_a + d_b) of the proof of Theorem 2, which keeps
                           w_ab + w_ba in its own coordinate and the internal weight in its
                           degree.  0: each level scores the coarse graph G_c as it is, without
                           the internal weight.                                             */
    int32_t reorder;    /* adjacency reordering (spc_coarsen only; the paper's closing section
                           suggests it).  1: the graph is first renumbered by (L_8(x), L_2(x),
                           x), where L_k(x) is the smallest node id within k hops of x, and
                           coarsened in that numbering: node x is node perm[x] there
                           (spc_get_reorder).  lift_out stays in the caller's numbering; the
                           retained levels and spc_take_result's coarse graph and edge map
                           refer to the renumbered graph, whose edge ids and whose order of
                           equal scores differ from the caller's.  0 (default): no reordering. */
} spc_options;

/* Per-level results retained by the context after spc_coarsen / spc_coarsen_batched /
 * spc_contract.  All pointers are device pointers owned by the context, valid until the next
 * coarsening call on the context or its destruction.  Level l maps the level-l input graph
 * (level 0 = the caller's graph) onto the level-l coarse graph.                            */
typedef struct {
    int64_t n;              /* nodes of this level's input graph                         */
    int64_t m;              /* undirected edges of this level's input graph               */
    int64_t n_c;            /* super-nodes produced                                       */
    int64_t m_c;            /* coarse undirected edges                                    */
    int64_t m_inter;        /* fine edges joining two different super-nodes               */
    int32_t status;         /* SPC_OK or SPC_WARN_TARGET_NOT_REACHED for this level        */
    spc_dtype wtype;        /* weight type of both graphs                                 */
    const void* score;      /* [m]   f per fine edge, binary64 or binary32 (scoretype)     */
    spc_dtype scoretype;    /* SPC_F64 or SPC_F32                                         */
    const int32_t* lift;    /* [n]   super-node of every fine node                        */
    const int32_t* emap;    /* [m]   coarse undirected edge of every fine edge, -1 inside  */
    const void* self_mass;  /* [n_c] weight inside every super-node (int64 for SPC_I32)    */
    const void* a_und;      /* [m_c] coarse undirected weights, coarse edge id order       */
    const int64_t* rowptr_c;/* [n_c+1] coarse CSR                                         */
    const int32_t* col_c;   /* [2 m_c]                                                    */
    const void* w_c;        /* [2 m_c]                                                    */
    const int32_t* perm;    /* [m_inter] inter-super-node fine edges sorted by (coarse edge,
                               fine edge)                                                 */
    const int32_t* seg;     /* [m_c+1] perm[seg[k] .. seg[k+1]) are coarse edge k's edges   */
    const int64_t* graph_ptr_c; /* [B+1] super-node offsets per graph (batched calls), else NULL */
    float ms;               /* device time of the level in milliseconds (CUDA events), or -1 */
    const void* mass;       /* [n_c] accumulated internal weight of every super-node: the
                               weight of the caller's edges inside it, as the self-mass reading
                               carries it (int64 for SPC_I32); NULL when the call did not use
                               that reading                                               */
} spc_level;

typedef struct spc_context spc_context;

/* ---- context ---------------------------------------------------------------------------- */

/* Create a context on the current CUDA device.  `stream` is a cudaStream_t (NULL: the legacy
 * default stream).  `allocator` may be NULL (cudaMalloc).  The context owns its workspace,
 * its captured CUDA graphs and the retained per-level results. */
SPC_API spc_status spc_context_create(spc_context** out, const spc_allocator* allocator, void* stream);

/* Destroy a context and free everything it owns.  NULL is accepted. */
SPC_API void spc_context_destroy(spc_context* ctx);

/* Bound every device-side wait and retry loop of later calls on the context (the look-back
 * of the scans and sorts, the union-find walks of the merge selection) to `iterations`;
 * 0 restores the default of 2^22.  A wait that reaches the bound gives up and the call returns
 * SPC_ERR_TIMEOUT; every index stays in range when a wait gives up, so the context stays
 * usable.  Meant for exercising the timeout path: a small bound makes waits give up. */
SPC_API spc_status spc_context_set_wait_limit(spc_context* ctx, uint32_t iterations);

/* Change the stream later calls are issued on (captured graphs are re-captured). */
SPC_API spc_status spc_context_set_stream(spc_context* ctx, void* stream);

/* Human-readable name of a status code (static storage). */
SPC_API const char* spc_status_string(spc_status status);

/* Default options: levels 1, validate 1, use_graph 1, schedule 0, self_mass 1, reorder 0. */
SPC_API spc_options spc_default_options(void);

/* ---- the full method ---------------------------------------------------------------------- */

/* Coarsen g to n_c super-nodes (Algorithm 1, repeated per options->levels).
 *   lift_out[n]     super-node (at the last level) of every node of g, ids ordered by smallest
 *                   member node id (device or host pointer, caller-allocated)
 *   n_c_actual      number of super-nodes at the last level (host pointer, may be NULL)
 * Per-level results (scores, maps, coarse graphs) are retained; see spc_get_level.  The last
 * level's coarse graph is the coarsened graph G_c (without diagonal entries: the weight inside
 * each super-node is its self-mass, and with options->self_mass its accumulated mass).
 * n_c >= n returns the identity.
 * Returns SPC_WARN_TARGET_NOT_REACHED if some level had more connected components than its
 * target. */
SPC_API spc_status spc_coarsen(spc_context* ctx, const spc_csr* g, int64_t n_c, const spc_options* options,
                       int32_t* lift_out, int64_t* n_c_actual);

/* Batched coarsening of B independent graphs stored as one block-diagonal CSR: graph b owns
 * nodes [graph_ptr[b], graph_ptr[b+1]) and has edges only among them.  Graph b is coarsened
 * to its own targets: max(1, floor(n_b / ratio)) at the last level, with `levels` halving
 * levels as in spc_options (ratio must then be 2^levels).  All graphs are processed by the
 * same kernel launches (no per-graph launches).
 *   graph_ptr[B+1]    int64, device or host
 *   lift_out[n]       global super-node ids; graph b's super-nodes are
 *                     [graph_ptr_c_out[b], graph_ptr_c_out[b+1])
 *   graph_ptr_c_out[B+1] int64 (device or host, may be NULL) */
SPC_API spc_status spc_coarsen_batched(spc_context* ctx, const spc_csr* g, const int64_t* graph_ptr,
                               int64_t B, int64_t ratio, const spc_options* options,
                               int32_t* lift_out, int64_t* graph_ptr_c_out);

/* The renumbering of the last spc_coarsen call made with options->reorder:
 * perm_out[x] (int32, n entries, device or host) = the id of node x in the renumbered graph.
 * SPC_ERR_INVALID_ARG when the last coarsening call did not reorder. */
SPC_API spc_status spc_get_reorder(spc_context* ctx, int32_t* perm_out);

/* Number of levels retained by the last coarsening call, and access to one of them. */
SPC_API int32_t spc_level_count(const spc_context* ctx);
SPC_API spc_status spc_get_level(const spc_context* ctx, int32_t level, spc_level* out);

/* The result of the last spc_coarsen / spc_coarsen_batched call in buffers the caller owns:
 * unlike the retained levels (spc_get_level), they outlive later calls on the context, so a
 * caller can hold several coarsenings at once (a pooling layer keeps one per graph).  Every
 * buffer is device memory allocated through the context's allocator (the spc_allocator given
 * to spc_context_create, else cudaMalloc); release them with spc_result_free (or that
 * allocator's free). */
typedef struct {
    int64_t n, m;        /* nodes and undirected edges of the caller's graph              */
    int64_t n_c, m_c;    /* super-nodes and coarse undirected edges of the last level      */
    spc_dtype wtype;     /* weight type                                                    */
    int32_t* lift;       /* [n]       super-node of every node (as lift_out)                */
    int32_t* emap;       /* [m]       coarse edge of every fine edge, -1 inside a super-node */
    int64_t* rowptr_c;   /* [n_c + 1] the coarse graph G_c (symmetric CSR, no diagonal)     */
    int32_t* col_c;      /* [2 m_c]                                                         */
    void* w_c;           /* [2 m_c]   of type wtype                                         */
    void* mass;          /* [n_c]     weight of the caller's edges inside every super-node as
                            the self-mass reading carries it (int64 for SPC_I32); NULL when
                            the call did not use that reading                             */
} spc_result;

/* Fill *out with the last coarsening's result (see spc_result).  SPC_ERR_INVALID_ARG when the
 * context holds no coarsening result; SPC_ERR_OOM (nothing kept) when an allocation fails. */
SPC_API spc_status spc_take_result(spc_context* ctx, spc_result* out);

/* Release the buffers of a result taken from this context and zero *r.  NULL is accepted. */
SPC_API void spc_result_free(spc_context* ctx, spc_result* r);

/* Copy `bytes` from src to dst on the context's stream and wait for it.  Either side may be
 * host or device memory; used to read retained results into caller buffers. */
SPC_API spc_status spc_copy(spc_context* ctx, void* dst, const void* src, size_t bytes);

/* ---- single steps (the same kernels spc_coarsen runs) ------------------------------------- */

/* S0-S3: validate g, weighted degrees, normalised rows, and the score of every undirected
 * edge in eid order (Theorem 1; Algorithm 1 fitness loop).  f_out[m] is binary64 for
 * SPC_I32/SPC_F64 and binary32 for SPC_F32.  *m_out (host, may be NULL) receives m. */
SPC_API spc_status spc_score(spc_context* ctx, const spc_csr* g, void* f_out, int64_t* m_out);

/* S4: edge ids sorted by (f, eid) ascending (Algorithm 1's sort; ties by node id).
 * f[m] of type ftype (SPC_F32 or SPC_F64, values >= +0); order_out[m] int32. */
SPC_API spc_status spc_sort_fitness(spc_context* ctx, int64_t m, const void* f, spc_dtype ftype,
                            int32_t* order_out);

/* S5-S6: the merge loop of Algorithm 1 given scores f[m] (as produced by spc_score): the
 * partition reached by merging in (f, eid) order until n_c super-nodes remain, and its
 * canonical lift (ids by smallest member).  merged_out[m] (uint8, may be NULL) marks the edges
 * that performed a merge. */
SPC_API spc_status spc_select_merges(spc_context* ctx, const spc_csr* g, const void* f, int64_t n_c,
                             int32_t* lift_out, uint8_t* merged_out, int64_t* n_c_actual);

/* S7: contract g by a given lift (values in [0, n_c), every id used) -- Definition 1.
 * Results are retained as level 0 (spc_get_level); *m_c_out (host, may be NULL) gets m_c.
 * Returns SPC_ERR_OVERFLOW if an SPC_I32 coarse weight exceeds int32. */
SPC_API spc_status spc_contract(spc_context* ctx, const spc_csr* g, const int32_t* lift, int64_t n_c,
                        int64_t* m_c_out);

/* S7 weights only, the assignment held fixed: a_und[k] = sum over perm[seg[k] .. seg[k+1]) of
 * w_und[e], summed in that (ascending eid) order.  w_und[m] and a_und[m_c] of type wtype
 * (SPC_F32 or SPC_F64), perm/seg as retained by a contraction.  Device pointers. */
SPC_API spc_status spc_contract_forward(spc_context* ctx, const int32_t* perm, const int32_t* seg,
                                int64_t m_c, const void* w_und, spc_dtype wtype, void* a_und);

/* S9: gradient of the weight contraction with the assignment held fixed:
 * grad_w[e] = grad_a[emap[e]] when emap[e] >= 0, else 0.  emap[m] int32; grad_a[m_c] and
 * grad_w[m] of type dtype (SPC_F32 or SPC_F64).  Device pointers. */
SPC_API spc_status spc_contract_backward(spc_context* ctx, const int32_t* emap, int64_t m,
                                 const void* grad_a, void* grad_w, spc_dtype dtype);

/* Fine edge -> last-level coarse edge through all retained levels (-1 once inside a
 * super-node).  emap_out[m of level 0] int32, device or host. */
SPC_API spc_status spc_compose_emap(spc_context* ctx, int32_t* emap_out);

/* ---- allocation-free variant ---------------------------------------------------------------- */

/* spc_sort_fitness without a context and without allocating: for callers that must not call
 * cudaMalloc (a fixed memory budget owned by another framework, threads that cannot take
 * cudaMalloc's implicit device synchronisation, memory reserved entirely up front).  The paper
 * has no counterpart; it is the S4 sort of spc_sort_fitness with its temporaries in one
 * file-scope device array of the library (22 MiB, held on every GPU that loads the library).
 *   m           number of scores, 0 <= m <= 2^20 (larger: SPC_ERR_TOO_LARGE, nothing launched)
 *   f           device pointer, m scores of type ftype (SPC_F32 or SPC_F64), values >= +0
 *   order_out   device pointer, m int32: edge ids sorted by (f, eid), the same result as
 *               spc_sort_fitness
 *   stream      cudaStream_t the work is enqueued on (NULL: legacy default stream)
 * Returns once the work is enqueued; the result is ready when the stream reaches it.  Host
 * pointers, and device memory of a GPU other than the current one, are rejected with
 * SPC_ERR_INVALID_ARG (staging them would need memory).  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress) for that device;
 * make it before any stream capture.  All calls share the array: calls that may execute
 * concurrently on the GPU race and must be ordered by the caller. */
SPC_API spc_status spc_sort_fitness_static(int64_t m, const void* f, spc_dtype ftype,
                                           int32_t* order_out, void* stream);

/* ---- node-feature pooling (graph-pooling layer on the coarsening) -------------------------- */

/* Mean of every super-node's member features.  Definition 2's lift averages over the member
 * pairs of two super-nodes (it divides by |u_c| |v_c|); for node features the same averaging
 * is the mean over members:
 *   xc[U][f] = (sum over the members v of U, in ascending v, of x[v][f]) / |U|
 * summed left to right in the feature type, then one IEEE division by |U|; 0 for a super-node
 * without members.
 *   lift[n]      int32 super-node of every node, values in [0, n_c) (e.g. a composed lift)
 *   x[n * F]     features, row-major, dtype SPC_F32 or SPC_F64
 *   xc_out[n_c * F]  result, row-major, same dtype
 * Device pointers, owned by the caller.  A lift value outside [0, n_c) returns
 * SPC_ERR_INVALID_ARG with xc_out unspecified. */
SPC_API spc_status spc_pool_features(spc_context* ctx, int64_t n, const int32_t* lift, int64_t n_c,
                                     int64_t F, spc_dtype dtype, const void* x, void* xc_out);

/* Gradient of spc_pool_features with the lift held fixed:
 *   grad_x[v][f] = grad_xc[lift[v]][f] / |lift[v]|   (one IEEE division).
 * grad_xc[n_c * F] and grad_x_out[n * F] row-major, dtype SPC_F32 or SPC_F64, device
 * pointers.  Errors as spc_pool_features. */
SPC_API spc_status spc_pool_features_backward(spc_context* ctx, int64_t n, const int32_t* lift,
                                              int64_t n_c, int64_t F, spc_dtype dtype,
                                              const void* grad_xc, void* grad_x_out);

/* ---- timing ------------------------------------------------------------------------------- */

/* Record CUDA events around every launch of the kernels whose name contains `kernel_substr`
 * ("*": every kernel; NULL or "" switches it off); spc_kernel_time returns the launches seen and their summed
 * device time since the last call to spc_time_kernel. */
SPC_API spc_status spc_time_kernel(spc_context* ctx, const char* kernel_substr);
SPC_API spc_status spc_kernel_time(spc_context* ctx, int64_t* launches, double* total_ms);

/* Per-kernel breakdown of the timed launches since the last spc_time_kernel: one line per
 * kernel, "name<TAB>launches<TAB>total_ms<TAB>bytes<TAB>fp_ops<LF>", NUL-terminated in
 * buf[len].  bytes is the sum over those launches of each launch's algorithmic DRAM bytes
 * (every input the operation needs read once, every output written once), 0 for launches
 * without such a model.  fp_ops, for the score kernels, is the arithmetic the score needs:
 * one addition per coordinate of N(a) u N(b) and one subtraction per coordinate in both rows,
 * summed over the timed launches (0 for other kernels).  Returns SPC_ERR_INVALID_ARG (with the
 * text truncated) if len is too small. */
SPC_API spc_status spc_kernel_profile(spc_context* ctx, char* buf, size_t len);

/* Number of kernel launches issued by the context since it was created (replayed graph
 * launches count their kernel nodes); 0 for a NULL context. */
SPC_API int64_t spc_launch_count(const spc_context* ctx);

/* 1 if the last spc_coarsen or spc_coarsen_batched call was served by replaying the captured
 * graph of the previous identical call (same sizes, same input checksum, and every logged
 * size confirmed on the device), 0 if it ran host-driven or ctx is NULL. */
SPC_API int spc_last_call_replayed(const spc_context* ctx);

#ifdef __cplusplus
}
#endif

#endif /* SPCOARSEN_H */
