/*
 * CPU oracle for sparse symbolic LU factorisation (gSoFa, Gaihre, Li, Liu,
 * arXiv 2007.00840).  TEST INFRASTRUCTURE ONLY: the library never links,
 * calls or falls back to this file.  Only the tests, the smoke check and the
 * CPU baseline leg of the benchmark use it.
 *
 * What it computes (Theorem 1, the fill-path theorem of Rose and Tarjan,
 * quoted in Section 2.1): entry (i, j) of L+U is nonzero iff j == i, or
 * A(i, j) != 0, or there is a directed path i -> ... -> j in G(A) whose
 * intermediate vertices are all numbered below min(i, j).
 *
 * How (Section 2.1, the fill2 algorithm, and Section 8, which relates fill2
 * to Dijkstra's algorithm with "the largest vertex on the path" as the
 * distance): for row i, let lab(w) be the smallest possible largest
 * intermediate vertex over all paths i -> w that only pass through vertices
 * below i (a minimax path label).  Direct neighbours have no intermediate
 * and get lab = -1.  Then
 *     j <  i is in L(i,:)  iff  lab(j) < j
 *     j >  i is in U(i,:)  iff  lab(j) < i   (i.e. j was reached at all)
 *     U(i,i) is always present (no pivoting, nonzero pivots).
 * lab is computed with a binary-heap Dijkstra whose path metric is
 * max(lab(v), v) for the step v -> w; the metric never decreases along a
 * path, so each vertex is final when it is popped.  Only vertices v < i are
 * expanded (they may act as intermediates); vertices above i are endpoints.
 *
 * The oracle also counts, per row, the vertices it expanded (V_scan) and the
 * adjacency entries it read (E_scan): the minimum work of a fill-path search
 * for that row.
 *
 * Supernodes (Definition 1, T3, Section 2.2; chunked as in Section 5):
 * scanning rows left to right, row s joins the supernode that starts at row r
 * and ends at s-1 iff nnz(U(s,:)) == nnz(U(s-1,:)) - 1 and L(s, r) != 0;
 * otherwise s starts a new supernode.  Every row that is a multiple of the
 * chunk size (the maximum supernode size, 128 by default) starts a new one.
 *
 * Build: gcc -O2 -fPIC -shared -pthread oracle.c -o liboracle.so
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define LAB_INF INT32_MAX

/* ---------------------------------------------------------------- heap -- */
typedef struct { int32_t key; int32_t v; } hent;
typedef struct { hent *a; int64_t size, cap; } heap_t;

static int heap_push(heap_t *h, int32_t key, int32_t v) {
    if (h->size == h->cap) {
        int64_t nc = h->cap ? 2 * h->cap : 1024;
        hent *na = (hent *)realloc(h->a, (size_t)nc * sizeof(hent));
        if (!na) return -1;
        h->a = na; h->cap = nc;
    }
    int64_t k = h->size++;
    while (k > 0) {
        int64_t p = (k - 1) / 2;
        if (h->a[p].key <= key) break;
        h->a[k] = h->a[p];
        k = p;
    }
    h->a[k].key = key; h->a[k].v = v;
    return 0;
}

static hent heap_pop(heap_t *h) {
    hent top = h->a[0];
    hent last = h->a[--h->size];
    int64_t k = 0;
    for (;;) {
        int64_t c = 2 * k + 1;
        if (c >= h->size) break;
        if (c + 1 < h->size && h->a[c + 1].key < h->a[c].key) c++;
        if (last.key <= h->a[c].key) break;
        h->a[k] = h->a[c];
        k = c;
    }
    if (h->size > 0) h->a[k] = last;
    return top;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* ------------------------------------------------------ per-row search -- */
typedef struct {
    int32_t *lab;      /* n entries, LAB_INF between rows */
    int32_t *touched;  /* vertices whose lab was set for this row */
    int64_t ntouched;
    heap_t heap;
} workspace;

typedef struct {
    int32_t nL, nU;
    int32_t *cols;     /* nL sorted L columns followed by nU sorted U columns */
    int64_t vscan, escan;
} row_result;

/* Minimax-label search for row i; fills *res.  Returns 0 or -1 on OOM. */
static int oracle_row(int32_t n, const int32_t *rowptr, const int32_t *colidx,
                      int32_t i, workspace *ws, row_result *res) {
    int32_t *lab = ws->lab;
    ws->ntouched = 0;
    ws->heap.size = 0;
    int64_t vscan = 0, escan = 0;

    /* direct neighbours: no intermediate vertex, label -1 */
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
        int32_t w = colidx[e];
        if (w == i) continue;
        if (lab[w] == LAB_INF) ws->touched[ws->ntouched++] = w;
        lab[w] = -1;
        if (heap_push(&ws->heap, -1, w)) return -1;
    }
    while (ws->heap.size > 0) {
        hent t = heap_pop(&ws->heap);
        int32_t v = t.v;
        if (t.key != lab[v]) continue;      /* stale entry */
        if (v > i) continue;                /* endpoint only, never an intermediate */
        vscan++;
        int32_t c = lab[v] > v ? lab[v] : v; /* largest intermediate if we pass v */
        for (int32_t e = rowptr[v]; e < rowptr[v + 1]; e++) {
            int32_t w = colidx[e];
            escan++;
            if (w == i) continue;
            if (c < lab[w]) {
                if (lab[w] == LAB_INF) ws->touched[ws->ntouched++] = w;
                lab[w] = c;
                if (heap_push(&ws->heap, c, w)) return -1;
            }
        }
    }
    /* collect L and U (diagonal always in U) */
    int32_t nL = 0, nU = 1;
    for (int64_t t = 0; t < ws->ntouched; t++) {
        int32_t w = ws->touched[t];
        if (w < i) { if (lab[w] < w) nL++; }
        else if (w > i) nU++;           /* any reached w > i has lab < i */
    }
    int32_t *cols = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nL + nU));
    if (!cols) return -1;
    int32_t a = 0, b = nL;
    cols[b++] = i;
    for (int64_t t = 0; t < ws->ntouched; t++) {
        int32_t w = ws->touched[t];
        if (w < i) { if (lab[w] < w) cols[a++] = w; }
        else if (w > i) cols[b++] = w;
        lab[w] = LAB_INF;
    }
    qsort(cols, (size_t)nL, sizeof(int32_t), cmp_i32);
    qsort(cols + nL, (size_t)nU, sizeof(int32_t), cmp_i32);
    res->nL = nL; res->nU = nU; res->cols = cols;
    res->vscan = vscan; res->escan = escan;
    return 0;
}

/* ---------------------------------------------------------- threading -- */
typedef struct {
    int32_t n; const int32_t *rowptr, *colidx;
    int32_t nrows; const int32_t *rows;
    row_result *res;
    int64_t next;            /* shared work counter */
    pthread_mutex_t mu;
    int err;
} job_t;

static void *worker(void *arg) {
    job_t *J = (job_t *)arg;
    workspace ws;
    ws.lab = (int32_t *)malloc(sizeof(int32_t) * (size_t)(J->n > 0 ? J->n : 1));
    ws.touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)(J->n > 0 ? J->n : 1));
    ws.heap.a = NULL; ws.heap.size = ws.heap.cap = 0;
    if (!ws.lab || !ws.touched) { J->err = -1; free(ws.lab); free(ws.touched); return NULL; }
    for (int32_t v = 0; v < J->n; v++) ws.lab[v] = LAB_INF;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int64_t k = J->next;
        J->next += 16;
        pthread_mutex_unlock(&J->mu);
        if (k >= J->nrows) break;
        int64_t e = k + 16 < J->nrows ? k + 16 : J->nrows;
        for (int64_t q = k; q < e; q++) {
            if (oracle_row(J->n, J->rowptr, J->colidx, J->rows[q], &ws, &J->res[q])) {
                J->err = -1;
            }
        }
    }
    free(ws.lab); free(ws.touched); free(ws.heap.a);
    return NULL;
}

typedef struct {
    int32_t nrows;
    row_result *res;
} oracle_handle;

/* Run the per-row search for rows[0..nrows) on nthreads threads (>= 1).
 * Returns an opaque handle (NULL on failure). */
void *oracle_run(int32_t n, const int32_t *rowptr, const int32_t *colidx,
                 int32_t nrows, const int32_t *rows, int32_t nthreads) {
    if (nthreads < 1) nthreads = 1;
    oracle_handle *H = (oracle_handle *)calloc(1, sizeof(oracle_handle));
    if (!H) return NULL;
    H->nrows = nrows;
    H->res = (row_result *)calloc((size_t)(nrows > 0 ? nrows : 1), sizeof(row_result));
    if (!H->res) { free(H); return NULL; }
    job_t J;
    J.n = n; J.rowptr = rowptr; J.colidx = colidx; J.nrows = nrows; J.rows = rows;
    J.res = H->res; J.next = 0; J.err = 0;
    pthread_mutex_init(&J.mu, NULL);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    int started = 0;
    for (int t = 0; t < nthreads; t++)
        if (pthread_create(&th[t], NULL, worker, &J) == 0) started++;
        else break;
    if (started == 0) worker(&J);
    for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&J.mu);
    if (J.err) {
        for (int32_t q = 0; q < nrows; q++) free(H->res[q].cols);
        free(H->res); free(H);
        return NULL;
    }
    return H;
}

/* Per-row counts and scan statistics (arrays of nrows). */
void oracle_counts(void *h, int32_t *nnzL, int32_t *nnzU, int64_t *vscan, int64_t *escan) {
    oracle_handle *H = (oracle_handle *)h;
    for (int32_t q = 0; q < H->nrows; q++) {
        if (nnzL) nnzL[q] = H->res[q].nL;
        if (nnzU) nnzU[q] = H->res[q].nU;
        if (vscan) vscan[q] = H->res[q].vscan;
        if (escan) escan[q] = H->res[q].escan;
    }
}

/* Concatenate the rows (in the order they were requested) into CSR arrays.
 * Lptr/Uptr have nrows+1 entries; Lcol/Ucol are sized by the counts. */
void oracle_rows(void *h, int64_t *Lptr, int32_t *Lcol, int64_t *Uptr, int32_t *Ucol) {
    oracle_handle *H = (oracle_handle *)h;
    int64_t a = 0, b = 0;
    Lptr[0] = 0; Uptr[0] = 0;
    for (int32_t q = 0; q < H->nrows; q++) {
        row_result *r = &H->res[q];
        memcpy(Lcol + a, r->cols, sizeof(int32_t) * (size_t)r->nL);
        memcpy(Ucol + b, r->cols + r->nL, sizeof(int32_t) * (size_t)r->nU);
        a += r->nL; b += r->nU;
        Lptr[q + 1] = a; Uptr[q + 1] = b;
    }
}

void oracle_free(void *h) {
    oracle_handle *H = (oracle_handle *)h;
    if (!H) return;
    for (int32_t q = 0; q < H->nrows; q++) free(H->res[q].cols);
    free(H->res);
    free(H);
}

/* ----------------------------------------------------------- supernodes -- */
/* Is column c present in the sorted L row s? (linear scan: plain, obviously correct) */
static int l_has(const int64_t *Lptr, const int32_t *Lcol, int32_t s, int32_t c) {
    for (int64_t e = Lptr[s]; e < Lptr[s + 1]; e++)
        if (Lcol[e] == c) return 1;
    return 0;
}

/* Greedy left-to-right T3 partition.  super_start receives the first row of
 * every supernode followed by n; returns the number of supernodes. */
int32_t oracle_supernodes(int32_t n, const int32_t *nnzU, const int64_t *Lptr,
                          const int32_t *Lcol, int32_t chunk, int32_t *super_start) {
    int32_t ns = 0;
    int32_t r = 0;
    for (int32_t s = 0; s < n; s++) {
        int join = 0;
        if (s > 0 && (chunk <= 0 || s % chunk != 0)) {
            join = (nnzU[s] == nnzU[s - 1] - 1) && l_has(Lptr, Lcol, s, r);
        }
        if (!join) { super_start[ns++] = s; r = s; }
    }
    super_start[ns] = n;
    return ns;
}
