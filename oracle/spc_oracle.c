/*
 * CPU oracle for spectral-bound greedy coarsening (Brissette, Huang, Slota, arXiv 2204.11757).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, sequential, obviously-correct statement of
 * what the GPU library computes.  Only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  It shares no code, header, table or helper with the CUDA library,
 * and the CUDA library never calls it.
 *
 * Build: cc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC [-fopenmp] (no FMA contraction, IEEE
 * binary32/binary64 with round-to-nearest; there are no multiplications in the arithmetic below,
 * only additions, subtractions, absolute values and divisions).
 *
 * What each function follows:
 *   orc_degree      Section 1, Theorem 1 and the sentence after it: d_x is the degree of x,
 *                   read as the weighted degree sum_y w_xy, summed in ascending y.
 *   orc_normalise   Theorem 1: the normalised adjacency vector w_x / d_x, one IEEE division per
 *                   stored entry.
 *   orc_score       Algorithm 1 (fitness loop) and Section 2 (one 1-norm per edge, cost
 *                   O(d_u + d_v)): f(a,b) = || w_a/d_a - w_b/d_b ||_1 over the full n-vectors,
 *                   i.e. over the sorted union N(a) u N(b), which contains a and b themselves
 *                   (coordinates b of row a and a of row b).  Summed in ascending coordinate
 *                   order, starting from 0.
 *   orc_score_parallel  the same scores with the edges split over the host's threads
 *                   (Algorithm 1's parallel fitness loop); a CPU baseline, same bits.
 *   orc_sort_fitness Algorithm 1 (sort of the fitness list): ascending f, ties by edge id.
 *   orc_greedy_merge Algorithm 1 (merge loop): walk the sorted list, merge the two super-nodes
 *                   of each edge unless they are already one, stop when n_c super-nodes remain
 *                   or the list is exhausted.  Scores are never recomputed (Section 2: the outer
 *                   loop of the explicit greedy algorithm is removed).
 *   orc_relabel     Definition 1 (super-nodes): super-node ids numbered by ascending smallest
 *                   member node id.
 *   orc_pool_features / orc_pool_backward  Definition 2's averaging over super-node sizes,
 *                   for node features: the mean over a super-node's members (ascending member
 *                   id, summed by a 256-ary tree of left-to-right sums), and its gradient with
 *                   the assignment held fixed.
 *   orc_contract    Definition 1: a_{v_c x} = sum over members v_i of w_{v_i x}, generalised to
 *                   pairs of super-nodes; edges inside one super-node leave the coarse graph and
 *                   their weight is reported as the super-node's self-mass (Definition 2 needs
 *                   it for the lift).  Coarse weights are summed over fine undirected edges in
 *                   ascending edge id.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_I32 = 0, ORC_F32 = 1, ORC_F64 = 2 };
enum { ORC_OK = 0, ORC_WARN_TARGET_NOT_REACHED = 1, ORC_ERR_ARG = -1, ORC_ERR_OVERFLOW = -8,
       ORC_ERR_NOMEM = -5 };

/* ---------------------------------------------------------------------------------------- */
/* S1: weighted degree, sequential in ascending column order.                                */
/* I32 weights -> int64 degree; F32 -> float; F64 -> double.                                 */
int orc_degree(int64_t n, const int64_t* rowptr, const void* w, int wtype, void* d_out)
{
    for (int64_t x = 0; x < n; ++x) {
        if (wtype == ORC_I32) {
            const int32_t* wi = (const int32_t*)w;
            int64_t s = 0;
            for (int64_t j = rowptr[x]; j < rowptr[x + 1]; ++j) s += (int64_t)wi[j];
            ((int64_t*)d_out)[x] = s;
        } else if (wtype == ORC_F32) {
            const float* wf = (const float*)w;
            float s = 0.0f;
            for (int64_t j = rowptr[x]; j < rowptr[x + 1]; ++j) s += wf[j];
            ((float*)d_out)[x] = s;
        } else if (wtype == ORC_F64) {
            const double* wd = (const double*)w;
            double s = 0.0;
            for (int64_t j = rowptr[x]; j < rowptr[x + 1]; ++j) s += wd[j];
            ((double*)d_out)[x] = s;
        } else {
            return ORC_ERR_ARG;
        }
    }
    return ORC_OK;
}

/* S2: p[j] = w[j] / d[row(j)] for every stored entry.  double for I32 and F64, float for F32. */
int orc_normalise(int64_t n, const int64_t* rowptr, const void* w, int wtype, const void* d,
                  void* p_out)
{
    for (int64_t x = 0; x < n; ++x) {
        for (int64_t j = rowptr[x]; j < rowptr[x + 1]; ++j) {
            if (wtype == ORC_I32) {
                double num = (double)((const int32_t*)w)[j];
                double den = (double)((const int64_t*)d)[x];
                ((double*)p_out)[j] = num / den;
            } else if (wtype == ORC_F32) {
                ((float*)p_out)[j] = ((const float*)w)[j] / ((const float*)d)[x];
            } else if (wtype == ORC_F64) {
                ((double*)p_out)[j] = ((const double*)w)[j] / ((const double*)d)[x];
            } else {
                return ORC_ERR_ARG;
            }
        }
    }
    return ORC_OK;
}

/* One 1-norm || p_a - p_b ||_1 by walking the two sorted rows in step.  A coordinate present
 * in one row only contributes |p - 0| = p; a coordinate in both contributes |p_a - p_b|. */
static double norm1_f64(const int32_t* col, const double* p, int64_t a0, int64_t a1, int64_t b0,
                        int64_t b1)
{
    double s = 0.0;
    int64_t i = a0, j = b0;
    while (i < a1 || j < b1) {
        double t;
        if (j >= b1 || (i < a1 && col[i] < col[j])) {
            t = p[i]; ++i;
        } else if (i >= a1 || col[j] < col[i]) {
            t = p[j]; ++j;
        } else {
            double diff = p[i] - p[j];
            t = diff < 0.0 ? -diff : diff;
            ++i; ++j;
        }
        s += t;
    }
    return s;
}

static float norm1_f32(const int32_t* col, const float* p, int64_t a0, int64_t a1, int64_t b0,
                       int64_t b1)
{
    float s = 0.0f;
    int64_t i = a0, j = b0;
    while (i < a1 || j < b1) {
        float t;
        if (j >= b1 || (i < a1 && col[i] < col[j])) {
            t = p[i]; ++i;
        } else if (i >= a1 || col[j] < col[i]) {
            t = p[j]; ++j;
        } else {
            float diff = p[i] - p[j];
            t = diff < 0.0f ? -diff : diff;
            ++i; ++j;
        }
        s += t;
    }
    return s;
}

/* S1-S3: f[eid] for every undirected edge (a, b), a < b, in edge-id order.
 * f is double for I32/F64 weights and float for F32 weights.  Returns the number of edges. */
int64_t orc_score(int64_t n, const int64_t* rowptr, const int32_t* col, const void* w, int wtype,
                  void* f_out)
{
    int64_t nnz = rowptr[n];
    size_t dsz = (wtype == ORC_F32) ? sizeof(float) : (wtype == ORC_I32 ? sizeof(int64_t)
                                                                       : sizeof(double));
    size_t psz = (wtype == ORC_F32) ? sizeof(float) : sizeof(double);
    void* d = malloc((size_t)(n > 0 ? n : 1) * dsz);
    void* p = malloc((size_t)(nnz > 0 ? nnz : 1) * psz);
    if (!d || !p) { free(d); free(p); return ORC_ERR_NOMEM; }
    int rc = orc_degree(n, rowptr, w, wtype, d);
    if (rc == ORC_OK) rc = orc_normalise(n, rowptr, w, wtype, d, p);
    if (rc != ORC_OK) { free(d); free(p); return rc; }
    int64_t e = 0;
    for (int64_t a = 0; a < n; ++a) {
        for (int64_t j = rowptr[a]; j < rowptr[a + 1]; ++j) {
            int64_t b = col[j];
            if (b <= a) continue;
            if (wtype == ORC_F32)
                ((float*)f_out)[e] = norm1_f32(col, (const float*)p, rowptr[a], rowptr[a + 1],
                                               rowptr[b], rowptr[b + 1]);
            else
                ((double*)f_out)[e] = norm1_f64(col, (const double*)p, rowptr[a], rowptr[a + 1],
                                                rowptr[b], rowptr[b + 1]);
            ++e;
        }
    }
    free(d); free(p);
    return e;
}

/* S1-S3 with the edges split evenly over the host's threads (OpenMP, static schedule): the
 * edge-partitioned parallel loop of Algorithm 1 on a CPU.  Every edge's norm is the same
 * sequential walk as in orc_score, so the scores are the same bits; only the edges are shared
 * out.  Used as a parallel CPU baseline.  Returns the number of edges; *threads_out is the
 * number of threads the loop ran on (1 without OpenMP). */
int64_t orc_score_parallel(int64_t n, const int64_t* rowptr, const int32_t* col, const void* w,
                           int wtype, void* f_out, int32_t* threads_out)
{
    int64_t nnz = rowptr[n];
    size_t dsz = (wtype == ORC_F32) ? sizeof(float) : (wtype == ORC_I32 ? sizeof(int64_t)
                                                                       : sizeof(double));
    size_t psz = (wtype == ORC_F32) ? sizeof(float) : sizeof(double);
    int64_t m = 0;
    for (int64_t a = 0; a < n; ++a)
        for (int64_t j = rowptr[a]; j < rowptr[a + 1]; ++j) m += col[j] > a ? 1 : 0;
    void* d = malloc((size_t)(n > 0 ? n : 1) * dsz);
    void* p = malloc((size_t)(nnz > 0 ? nnz : 1) * psz);
    int32_t* eu = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    int64_t* ej = (int64_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int64_t));
    if (!d || !p || !eu || !ej) { free(d); free(p); free(eu); free(ej); return ORC_ERR_NOMEM; }
    int rc = orc_degree(n, rowptr, w, wtype, d);
    if (rc == ORC_OK) rc = orc_normalise(n, rowptr, w, wtype, d, p);
    if (rc != ORC_OK) { free(d); free(p); free(eu); free(ej); return rc; }
    int64_t e = 0;
    for (int64_t a = 0; a < n; ++a)
        for (int64_t j = rowptr[a]; j < rowptr[a + 1]; ++j)
            if (col[j] > a) { eu[e] = (int32_t)a; ej[e] = j; ++e; }
    int32_t threads = 1;
#ifdef _OPENMP
    threads = (int32_t)omp_get_max_threads();
#endif
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < m; ++k) {
        const int64_t a = eu[k], b = col[ej[k]];
        if (wtype == ORC_F32)
            ((float*)f_out)[k] = norm1_f32(col, (const float*)p, rowptr[a], rowptr[a + 1],
                                           rowptr[b], rowptr[b + 1]);
        else
            ((double*)f_out)[k] = norm1_f64(col, (const double*)p, rowptr[a], rowptr[a + 1],
                                            rowptr[b], rowptr[b + 1]);
    }
    if (threads_out) *threads_out = threads;
    free(d); free(p); free(eu); free(ej);
    return m;
}

/* ---------------------------------------------------------------------------------------- */
/* S4: sort the fitness list ascending, ties broken by edge id (lexicographic node-id order). */
static const void* g_sort_f;   /* qsort has no context argument; the oracle is single-threaded */
static int g_sort_ftype;

static int cmp_fitness(const void* x, const void* y)
{
    int32_t ex = *(const int32_t*)x, ey = *(const int32_t*)y;
    if (g_sort_ftype == ORC_F32) {
        float fx = ((const float*)g_sort_f)[ex], fy = ((const float*)g_sort_f)[ey];
        if (fx < fy) return -1;
        if (fx > fy) return 1;
    } else {
        double fx = ((const double*)g_sort_f)[ex], fy = ((const double*)g_sort_f)[ey];
        if (fx < fy) return -1;
        if (fx > fy) return 1;
    }
    return (ex < ey) ? -1 : (ex > ey);
}

int orc_sort_fitness(int64_t m, const void* f, int ftype, int32_t* order_out)
{
    for (int64_t e = 0; e < m; ++e) order_out[e] = (int32_t)e;
    g_sort_f = f;
    g_sort_ftype = ftype;
    qsort(order_out, (size_t)m, sizeof(int32_t), cmp_fitness);
    return ORC_OK;
}

/* ---------------------------------------------------------------------------------------- */
/* S5: the merge loop.  Super-node membership is tracked with a union-find forest (only which
 * nodes share a super-node matters here; the numbering is fixed by orc_relabel).            */
static int32_t uf_find(int32_t* parent, int32_t x)
{
    int32_t r = x;
    while (parent[r] != r) r = parent[r];
    while (parent[x] != r) { int32_t nx = parent[x]; parent[x] = r; x = nx; }
    return r;
}

/* rep_out[x] = smallest node id in x's super-node after the loop.
 * merged_out[e] (optional) = 1 if edge e caused a merge.  *s_out = super-node count.
 * Returns ORC_WARN_TARGET_NOT_REACHED if the list ran out with more than n_c super-nodes. */
int orc_greedy_merge(int64_t n, int64_t m, const int32_t* eu, const int32_t* ev,
                     const int32_t* order, int64_t n_c, int32_t* rep_out, uint8_t* merged_out,
                     int64_t* s_out)
{
    if (n_c < 1) return ORC_ERR_ARG;
    int32_t* parent = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!parent) return ORC_ERR_NOMEM;
    for (int64_t x = 0; x < n; ++x) parent[x] = (int32_t)x;
    if (merged_out) memset(merged_out, 0, (size_t)m);
    int64_t s = n;
    int64_t idx = 0;
    while (s > n_c && idx < m) {
        int32_t e = order[idx++];
        int32_t ra = uf_find(parent, eu[e]);
        int32_t rb = uf_find(parent, ev[e]);
        if (ra == rb) continue;           /* already one super-node: no merge, s unchanged */
        parent[rb] = ra;
        if (merged_out) merged_out[e] = 1;
        s -= 1;
    }
    /* smallest member of every super-node */
    int32_t* minmem = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!minmem) { free(parent); return ORC_ERR_NOMEM; }
    for (int64_t x = 0; x < n; ++x) minmem[x] = INT32_MAX;
    for (int64_t x = 0; x < n; ++x) {
        int32_t r = uf_find(parent, (int32_t)x);
        if ((int32_t)x < minmem[r]) minmem[r] = (int32_t)x;
    }
    for (int64_t x = 0; x < n; ++x) rep_out[x] = minmem[uf_find(parent, (int32_t)x)];
    free(minmem);
    free(parent);
    *s_out = s;
    return (s > n_c) ? ORC_WARN_TARGET_NOT_REACHED : ORC_OK;
}

/* S6: super-node id of x = number of distinct representatives smaller than rep[x].
 * rep[x] is the smallest member of x's super-node, so rep[r] == r marks one super-node each. */
int orc_relabel(int64_t n, const int32_t* rep, int32_t* lift_out, int64_t* n_c_out)
{
    int32_t* id = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!id) return ORC_ERR_NOMEM;
    int32_t next = 0;
    for (int64_t x = 0; x < n; ++x) {
        if (rep[x] == (int32_t)x) id[x] = next++;
        else id[x] = -1;
    }
    for (int64_t x = 0; x < n; ++x) lift_out[x] = id[rep[x]];
    free(id);
    *n_c_out = next;
    return ORC_OK;
}

/* ---------------------------------------------------------------------------------------- */
/* S7: contraction (Definition 1).                                                            */
typedef struct { int32_t lo, hi, e; } orc_triple;

static int cmp_triple(const void* x, const void* y)
{
    const orc_triple* a = (const orc_triple*)x;
    const orc_triple* b = (const orc_triple*)y;
    if (a->lo != b->lo) return a->lo < b->lo ? -1 : 1;
    if (a->hi != b->hi) return a->hi < b->hi ? -1 : 1;
    return (a->e < b->e) ? -1 : (a->e > b->e);
}

typedef struct { int32_t row, col; int64_t k; } orc_dir;

static int cmp_dir(const void* x, const void* y)
{
    const orc_dir* a = (const orc_dir*)x;
    const orc_dir* b = (const orc_dir*)y;
    if (a->row != b->row) return a->row < b->row ? -1 : 1;
    return (a->col < b->col) ? -1 : (a->col > b->col);
}

/* Inputs: the fine undirected edge list (eu < ev, edge-id order) with weights w_und, the lift
 * map c[n] with values in [0, n_c).
 * Outputs:
 *   emap[e]      coarse undirected edge id of fine edge e, or -1 when both ends share a
 *                super-node;
 *   self_mass[U] sum of the weights of fine edges inside super-node U, ascending edge id
 *                (int64 for I32 weights, float for F32, double for F64);
 *   a_und[k]     weight of coarse undirected edge k, k in lexicographic (U, V) order, U < V,
 *                summed over its fine edges in ascending edge id (same type as the input
 *                weights; I32 sums are exact in int64 and must fit in int32);
 *   rowptr_c[n_c+1], col_c[2 m_c], w_c[2 m_c]   the symmetric coarse CSR (rows by super-node
 *                id, ascending columns), w_c mirrors a_und;
 *   *m_c_out     number of coarse undirected edges.
 * a_und/col_c/w_c must hold at least m (>= m_c) entries; col_c/w_c 2m.                      */
int orc_contract(int64_t n, int64_t m, const int32_t* eu, const int32_t* ev, const void* w_und,
                 int wtype, const int32_t* c, int64_t n_c, int32_t* emap, void* self_mass,
                 void* a_und, int64_t* rowptr_c, int32_t* col_c, void* w_c, int64_t* m_c_out)
{
    (void)n;
    if (wtype == ORC_I32) memset(self_mass, 0, (size_t)n_c * sizeof(int64_t));
    else if (wtype == ORC_F32) { for (int64_t u = 0; u < n_c; ++u) ((float*)self_mass)[u] = 0.0f; }
    else if (wtype == ORC_F64) { for (int64_t u = 0; u < n_c; ++u) ((double*)self_mass)[u] = 0.0; }
    else return ORC_ERR_ARG;

    orc_triple* t = (orc_triple*)malloc((size_t)(m > 0 ? m : 1) * sizeof(orc_triple));
    if (!t) return ORC_ERR_NOMEM;
    int64_t nt = 0;
    for (int64_t e = 0; e < m; ++e) {
        int32_t U = c[eu[e]], V = c[ev[e]];
        if (U == V) {
            emap[e] = -1;
            if (wtype == ORC_I32) ((int64_t*)self_mass)[U] += ((const int32_t*)w_und)[e];
            else if (wtype == ORC_F32) ((float*)self_mass)[U] += ((const float*)w_und)[e];
            else ((double*)self_mass)[U] += ((const double*)w_und)[e];
            continue;
        }
        t[nt].lo = U < V ? U : V;
        t[nt].hi = U < V ? V : U;
        t[nt].e = (int32_t)e;
        ++nt;
    }
    qsort(t, (size_t)nt, sizeof(orc_triple), cmp_triple);

    int rc = ORC_OK;
    int64_t k = -1;
    int32_t* klo = (int32_t*)malloc((size_t)(nt > 0 ? nt : 1) * sizeof(int32_t));
    int32_t* khi = (int32_t*)malloc((size_t)(nt > 0 ? nt : 1) * sizeof(int32_t));
    if (!klo || !khi) { free(t); free(klo); free(khi); return ORC_ERR_NOMEM; }
    int64_t acc_i = 0; float acc_f = 0.0f; double acc_d = 0.0;
    for (int64_t i = 0; i < nt; ++i) {
        int new_run = (i == 0) || t[i].lo != t[i - 1].lo || t[i].hi != t[i - 1].hi;
        if (new_run) {
            if (k >= 0) {
                if (wtype == ORC_I32) {
                    if (acc_i > INT32_MAX) rc = ORC_ERR_OVERFLOW;
                    ((int32_t*)a_und)[k] = (int32_t)acc_i;
                } else if (wtype == ORC_F32) ((float*)a_und)[k] = acc_f;
                else ((double*)a_und)[k] = acc_d;
            }
            ++k;
            klo[k] = t[i].lo; khi[k] = t[i].hi;
            acc_i = 0; acc_f = 0.0f; acc_d = 0.0;
        }
        int32_t e = t[i].e;
        emap[e] = (int32_t)k;
        if (wtype == ORC_I32) acc_i += ((const int32_t*)w_und)[e];
        else if (wtype == ORC_F32) acc_f += ((const float*)w_und)[e];
        else acc_d += ((const double*)w_und)[e];
    }
    if (k >= 0) {
        if (wtype == ORC_I32) {
            if (acc_i > INT32_MAX) rc = ORC_ERR_OVERFLOW;
            ((int32_t*)a_und)[k] = (int32_t)acc_i;
        } else if (wtype == ORC_F32) ((float*)a_und)[k] = acc_f;
        else ((double*)a_und)[k] = acc_d;
    }
    int64_t m_c = k + 1;
    free(t);

    /* symmetric coarse CSR: both orientations of every coarse edge, sorted by (row, col) */
    orc_dir* dl = (orc_dir*)malloc((size_t)(2 * m_c > 0 ? 2 * m_c : 1) * sizeof(orc_dir));
    if (!dl) { free(klo); free(khi); return ORC_ERR_NOMEM; }
    for (int64_t q = 0; q < m_c; ++q) {
        dl[2 * q].row = klo[q]; dl[2 * q].col = khi[q]; dl[2 * q].k = q;
        dl[2 * q + 1].row = khi[q]; dl[2 * q + 1].col = klo[q]; dl[2 * q + 1].k = q;
    }
    qsort(dl, (size_t)(2 * m_c), sizeof(orc_dir), cmp_dir);
    for (int64_t u = 0; u <= n_c; ++u) rowptr_c[u] = 0;
    for (int64_t j = 0; j < 2 * m_c; ++j) rowptr_c[dl[j].row + 1] += 1;
    for (int64_t u = 0; u < n_c; ++u) rowptr_c[u + 1] += rowptr_c[u];
    for (int64_t j = 0; j < 2 * m_c; ++j) {
        col_c[j] = dl[j].col;
        if (wtype == ORC_I32) ((int32_t*)w_c)[j] = ((int32_t*)a_und)[dl[j].k];
        else if (wtype == ORC_F32) ((float*)w_c)[j] = ((float*)a_und)[dl[j].k];
        else ((double*)w_c)[j] = ((double*)a_und)[dl[j].k];
    }
    free(dl); free(klo); free(khi);
    *m_c_out = m_c;
    return rc;
}

/* S9 (reference gradient of the weight contraction with the assignment held fixed):
 * grad_w[e] = grad_a[emap[e]], or 0 when emap[e] == -1.  ftype F32 or F64. */
int orc_contract_backward(int64_t m, const int32_t* emap, const void* grad_a, int ftype,
                          void* grad_w)
{
    for (int64_t e = 0; e < m; ++e) {
        int32_t k = emap[e];
        if (ftype == ORC_F32) ((float*)grad_w)[e] = (k < 0) ? 0.0f : ((const float*)grad_a)[k];
        else if (ftype == ORC_F64) ((double*)grad_w)[e] = (k < 0) ? 0.0 : ((const double*)grad_a)[k];
        else return ORC_ERR_ARG;
    }
    return ORC_OK;
}

/* ---------------------------------------------------------------------------------------- */
/* Node-feature pooling onto the super-nodes and its gradient (a graph-pooling layer built on
 * the coarsening).  Definition 2's lift averages over the member pairs of two super-nodes
 * (divides by |u_c| |v_c|); its node counterpart is the mean over a super-node's members:
 *   xc[U][f] = S(x[v][f] for the members v of U in ascending v) / |U|.
 * The paper does not use node features, so the summation order S is this library's choice, a
 * 256-ary tree over the list:
 *   S(list) = ((0 + t_0) + t_1) + ... + t_(k-1)        if k <= ORC_POOL_CHUNK,
 *   S(list) = S([S(chunk_0), S(chunk_1), ...])          otherwise,
 * where chunk_i are the consecutive groups of ORC_POOL_CHUNK items; every addition in the
 * feature type; then one IEEE division by |U| (converted to the feature type).  x is n-by-F
 * row-major, xc n_c-by-F.  A super-node without members gets 0.
 * Gradient (lift held fixed): grad_x[v][f] = grad_xc[c(v)][f] / |c(v)|.                    */
#define ORC_POOL_CHUNK 256

static double pool_tree_f64(double* t, int64_t k)
{
    while (k > ORC_POOL_CHUNK) {  /* replace the list by its chunk sums, in place */
        int64_t m = 0;
        for (int64_t c = 0; c < k; c += ORC_POOL_CHUNK) {
            double s = 0.0;
            for (int64_t i = c; i < k && i < c + ORC_POOL_CHUNK; ++i) s = s + t[i];
            t[m++] = s;
        }
        k = m;
    }
    double s = 0.0;
    for (int64_t i = 0; i < k; ++i) s = s + t[i];
    return s;
}

static float pool_tree_f32(float* t, int64_t k)
{
    while (k > ORC_POOL_CHUNK) {
        int64_t m = 0;
        for (int64_t c = 0; c < k; c += ORC_POOL_CHUNK) {
            float s = 0.0f;
            for (int64_t i = c; i < k && i < c + ORC_POOL_CHUNK; ++i) s = s + t[i];
            t[m++] = s;
        }
        k = m;
    }
    float s = 0.0f;
    for (int64_t i = 0; i < k; ++i) s = s + t[i];
    return s;
}

static int64_t* pool_counts(int64_t n, const int32_t* lift, int64_t n_c)
{
    int64_t* cnt = (int64_t*)calloc((size_t)(n_c > 0 ? n_c : 1), sizeof(int64_t));
    if (!cnt) return NULL;
    for (int64_t v = 0; v < n; ++v) {
        if (lift[v] < 0 || lift[v] >= n_c) { free(cnt); return NULL; }
        cnt[lift[v]] += 1;
    }
    return cnt;
}

int orc_pool_features(int64_t n, const int32_t* lift, int64_t n_c, int64_t F, const void* x,
                      int ftype, void* xc_out)
{
    if (ftype != ORC_F32 && ftype != ORC_F64) return ORC_ERR_ARG;
    int64_t* cnt = pool_counts(n, lift, n_c);
    int64_t* start = (int64_t*)malloc((size_t)(n_c + 1) * sizeof(int64_t));
    int64_t* fill = (int64_t*)calloc((size_t)(n_c > 0 ? n_c : 1), sizeof(int64_t));
    int32_t* members = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    const size_t esz = ftype == ORC_F32 ? sizeof(float) : sizeof(double);
    void* t = malloc((size_t)(n > 0 ? n : 1) * esz);
    if (!cnt || !start || !fill || !members || !t) {
        free(cnt); free(start); free(fill); free(members); free(t);
        return ORC_ERR_ARG;
    }
    /* every super-node's members in ascending id */
    start[0] = 0;
    for (int64_t u = 0; u < n_c; ++u) start[u + 1] = start[u] + cnt[u];
    for (int64_t v = 0; v < n; ++v) members[start[lift[v]] + fill[lift[v]]++] = (int32_t)v;
    for (int64_t u = 0; u < n_c; ++u) {
        const int64_t k = cnt[u];
        for (int64_t f = 0; f < F; ++f) {
            if (ftype == ORC_F32) {
                float* tf = (float*)t;
                for (int64_t i = 0; i < k; ++i)
                    tf[i] = ((const float*)x)[members[start[u] + i] * F + f];
                ((float*)xc_out)[u * F + f] = k ? pool_tree_f32(tf, k) / (float)k : 0.0f;
            } else {
                double* td = (double*)t;
                for (int64_t i = 0; i < k; ++i)
                    td[i] = ((const double*)x)[members[start[u] + i] * F + f];
                ((double*)xc_out)[u * F + f] = k ? pool_tree_f64(td, k) / (double)k : 0.0;
            }
        }
    }
    free(cnt); free(start); free(fill); free(members); free(t);
    return ORC_OK;
}

int orc_pool_backward(int64_t n, const int32_t* lift, int64_t n_c, int64_t F,
                      const void* grad_xc, int ftype, void* grad_x)
{
    if (ftype != ORC_F32 && ftype != ORC_F64) return ORC_ERR_ARG;
    int64_t* cnt = pool_counts(n, lift, n_c);
    if (!cnt) return ORC_ERR_ARG;
    for (int64_t v = 0; v < n; ++v) {
        const int64_t u = lift[v];
        for (int64_t f = 0; f < F; ++f) {
            if (ftype == ORC_F32)
                ((float*)grad_x)[v * F + f] = ((const float*)grad_xc)[u * F + f] / (float)cnt[u];
            else
                ((double*)grad_x)[v * F + f] = ((const double*)grad_xc)[u * F + f] / (double)cnt[u];
        }
    }
    free(cnt);
    return ORC_OK;
}
