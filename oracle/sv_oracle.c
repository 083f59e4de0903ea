/*
 * FP64 CPU oracle: state-vector loops.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header or
 * constant with the CUDA path.
 *
 * A state is 2^n complex amplitudes stored as interleaved (re, im) doubles.
 * Wire w sits at bit (n - 1 - w) of an amplitude index: wire 0 is the most
 * significant bit (Alg. 1, q_offset = n - q - 1).
 *
 * The loops are deliberately plain: every index is visited and bits are tested
 * one by one; no masks are precomputed beyond the offsets of a gate's 2^k local
 * amplitudes.  Parallel loops only split independent groups over threads, so
 * results do not depend on the thread count; reductions use a fixed block
 * decomposition for the same reason (Sec. 4.2 reports equal outputs across runs).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_K 6
#define ORC_BLOCK 4096

static int bitpos(int n, int w) { return n - 1 - w; }

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/*
 * Apply a dense 2^k x 2^k complex matrix M (row-major, interleaved re/im) to
 * the target wires, on the groups whose control wires hold the given values.
 * Local index l of the matrix: bit (k-1-j) of l is the value of wires[j], so
 * wires[0] is the most significant local bit, matching the wire-0-is-MSB
 * convention of the whole state.  Controlled gates only touch the groups whose
 * control bits match (Alg. 2); all other amplitudes are left as they are.
 * Returns 0, or -1 on bad arguments.
 */
int orc_apply(double *psi, int n, int k, const int *wires, const double *M,
              int nc, const int *cwires, const int *cvals)
{
    if (k < 1 || k > ORC_MAX_K || n < k || n > 40) return -1;
    const int64_t N = (int64_t)1 << n;
    const int K = 1 << k;
    int64_t off[1 << ORC_MAX_K];
    int tpos[ORC_MAX_K];
    for (int j = 0; j < k; ++j) {
        if (wires[j] < 0 || wires[j] >= n) return -1;
        tpos[j] = bitpos(n, wires[j]);
    }
    for (int l = 0; l < K; ++l) {
        int64_t o = 0;
        for (int j = 0; j < k; ++j)
            if ((l >> (k - 1 - j)) & 1) o += (int64_t)1 << tpos[j];
        off[l] = o;
    }
    int cpos[64];
    for (int c = 0; c < nc; ++c) {
        if (cwires[c] < 0 || cwires[c] >= n) return -1;
        cpos[c] = bitpos(n, cwires[c]);
    }

#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < N; ++b) {
        int skip = 0;
        for (int j = 0; j < k && !skip; ++j)
            if ((b >> tpos[j]) & 1) skip = 1;          /* b must have every target bit 0 */
        for (int c = 0; c < nc && !skip; ++c)
            if (((b >> cpos[c]) & 1) != (cvals ? cvals[c] : 1)) skip = 1;
        if (skip) continue;
        double vr[1 << ORC_MAX_K], vi[1 << ORC_MAX_K];
        for (int l = 0; l < K; ++l) {
            vr[l] = psi[2 * (b + off[l])];
            vi[l] = psi[2 * (b + off[l]) + 1];
        }
        for (int r = 0; r < K; ++r) {
            double ar = 0.0, ai = 0.0;
            for (int c = 0; c < K; ++c) {
                const double mr = M[2 * (r * K + c)], mi = M[2 * (r * K + c) + 1];
                ar += mr * vr[c] - mi * vi[c];
                ai += mr * vi[c] + mi * vr[c];
            }
            psi[2 * (b + off[r])] = ar;
            psi[2 * (b + off[r]) + 1] = ai;
        }
    }
    return 0;
}

/* Zero every amplitude whose control wires do not hold the given values. */
int orc_project_controls(double *psi, int n, int nc, const int *cwires, const int *cvals)
{
    const int64_t N = (int64_t)1 << n;
    for (int c = 0; c < nc; ++c)
        if (cwires[c] < 0 || cwires[c] >= n) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        for (int c = 0; c < nc; ++c) {
            if (((i >> bitpos(n, cwires[c])) & 1) != (cvals ? cvals[c] : 1)) {
                psi[2 * i] = 0.0;
                psi[2 * i + 1] = 0.0;
                break;
            }
        }
    }
    return 0;
}

/*
 * out = sum_i conj(a_i) * b_i over 2^n amplitudes.  Fixed decomposition: each
 * block of ORC_BLOCK consecutive indices is summed in index order, then the
 * block sums are added in block order.  The result is the same for any number
 * of threads.
 */
void orc_inner(const double *a, const double *b, int n, double *out)
{
    const int64_t N = (int64_t)1 << n;
    const int64_t nb = (N + ORC_BLOCK - 1) / ORC_BLOCK;
    double *part = (double *)malloc(sizeof(double) * 2 * (size_t)nb);
#pragma omp parallel for schedule(static)
    for (int64_t blk = 0; blk < nb; ++blk) {
        double sr = 0.0, si = 0.0;
        const int64_t lo = blk * ORC_BLOCK;
        const int64_t hi = lo + ORC_BLOCK < N ? lo + ORC_BLOCK : N;
        for (int64_t i = lo; i < hi; ++i) {
            const double ar = a[2 * i], ai = a[2 * i + 1];
            const double br = b[2 * i], bi = b[2 * i + 1];
            sr += ar * br + ai * bi;
            si += ar * bi - ai * br;
        }
        part[2 * blk] = sr;
        part[2 * blk + 1] = si;
    }
    double sr = 0.0, si = 0.0;
    for (int64_t blk = 0; blk < nb; ++blk) {
        sr += part[2 * blk];
        si += part[2 * blk + 1];
    }
    free(part);
    out[0] = sr;
    out[1] = si;
}

/* y += (cr + i ci) * x over 2^n amplitudes. */
void orc_axpy(double *y, const double *x, int n, double cr, double ci)
{
    const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        const double xr = x[2 * i], xi = x[2 * i + 1];
        y[2 * i] += cr * xr - ci * xi;
        y[2 * i + 1] += cr * xi + ci * xr;
    }
}

/* dst = src over 2^n amplitudes. */
void orc_copy(double *dst, const double *src, int n)
{
    const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < 2 * N; ++i) dst[i] = src[i];
}

/* psi = |basis> */
void orc_basis(double *psi, int n, int64_t basis)
{
    const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < 2 * N; ++i) psi[i] = 0.0;
    psi[2 * basis] = 1.0;
}
