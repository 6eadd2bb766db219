/*
 * Parallel build of the FP64 oracle, used only to time the CPU baseline.
 *
 * TEST INFRASTRUCTURE ONLY, like pic_oracle.c, which this file includes
 * unchanged: every particle is pushed and deposited by the same code, but the
 * particles of a species are split into one contiguous block per OpenMP
 * thread.  Each thread deposits its block into current arrays of its own;
 * these are then added into the grid in thread order.  A run is therefore
 * deterministic for a given thread count and differs from the serial oracle
 * only in the order of the FP64 current sums and of the radiated-energy sum.
 * The field update stays serial (it is O(Nx) per step).
 */
#define OR_PARALLEL_PUSH 1
#include "pic_oracle.c"

#include <limits.h>
#include <omp.h>

/* Per-thread current arrays (Jx, Jy, Jz, each Nx + 1 + 2 OR_PAD), kept zero
 * between steps; grown on demand and held until the process exits. */
static double** g_tJ = NULL;
static size_t g_tlen = 0;
static int g_tn = 0;

int or_threads(void) { return omp_get_max_threads(); }

static int ensure_thread_buffers(int T, size_t len) {
    if (T <= g_tn && len <= g_tlen) return 0;
    for (int t = 0; t < g_tn; t++) free(g_tJ[t]);
    free(g_tJ);
    g_tJ = (double**)calloc((size_t)T, sizeof(double*));
    if (!g_tJ) return -1;
    for (int t = 0; t < T; t++) {
        g_tJ[t] = (double*)calloc(3 * len, sizeof(double));
        if (!g_tJ[t]) return -1;
    }
    g_tn = T;
    g_tlen = len;
    return 0;
}

static void push_species_parallel(or_sim* s, int k) {
    or_species* sp = &s->sp[k];
    const int T = omp_get_max_threads();
    const size_t len = (size_t)s->Nx + 1 + 2 * OR_PAD;
    if (T <= 1 || sp->n < 4096 || ensure_thread_buffers(T, len) != 0) {
        push_species(s, k);
        return;
    }
    double* urad = (double*)calloc((size_t)T, sizeof(double));
    int* lo = (int*)calloc((size_t)T, sizeof(int));
    int* hi = (int*)calloc((size_t)T, sizeof(int));
#pragma omp parallel num_threads(T)
    {
        const int t = omp_get_thread_num();
        const int64_t i0 = sp->n * t / T, i1 = sp->n * (t + 1) / T;
        /* cells this block can deposit to: a particle moves less than one cell
         * per step and touches at most cells floor(x) - 1 .. floor(x) + 2 */
        int a = INT_MAX, b = INT_MIN;
        for (int64_t i = i0; i < i1; i++) {
            const int c = (int)floor(sp->xi[i]);
            if (c < a) a = c;
            if (c > b) b = c;
        }
        or_sim loc = *s; /* fields shared (read only); current and radiated tally private */
        loc.Jx = g_tJ[t] + OR_PAD;
        loc.Jy = loc.Jx + len;
        loc.Jz = loc.Jy + len;
        loc.U_rad = 0.0;
        push_range(&loc, k, i0, i1);
        urad[t] = loc.U_rad;
        lo[t] = a - 1;
        hi[t] = b + 2;
    }
    for (int t = 0; t < T; t++) {
        if (lo[t] > hi[t]) continue; /* empty block */
        int a = lo[t] < -OR_PAD ? -OR_PAD : lo[t];
        int b = hi[t] > s->Nx + OR_PAD ? s->Nx + OR_PAD : hi[t];
        double* jx = g_tJ[t] + OR_PAD;
        double* jy = jx + len;
        double* jz = jy + len;
        for (int i = a; i <= b; i++) {
            s->Jx[i] += jx[i];
            s->Jy[i] += jy[i];
            s->Jz[i] += jz[i];
            jx[i] = jy[i] = jz[i] = 0.0;
        }
        s->U_rad += urad[t];
    }
    free(urad);
    free(lo);
    free(hi);
}
