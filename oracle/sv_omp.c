/*
 * Plain FP64 state-vector update in C, parallel over set ids with OpenMP.
 *
 * TEST INFRASTRUCTURE ONLY, like the rest of oracle/: only the tests, the
 * package entry's smoke check and the benchmark's CPU-baseline / reference
 * leg load it.  It shares no code, header or constant with the CUDA library.
 *
 * It computes exactly what oracle/statevector.py's apply_gate computes,
 * written as the loop of Section 3 ("Fast Schroedinger simulation"): a
 * k-qubit gate on qubits q_0..q_{k-1} splits the 2^n amplitudes into the
 * 2^(n-k) disjoint sets of 2^k amplitudes whose indices agree outside the
 * gate's qubits; the n-k remaining index bits, read in order, are the set
 * id s.  For every set:
 *   a[l] = psi[base(s) | sum_i bit(l, k-1-i) << q_i],   l < 2^k
 *   psi[same index of l] = sum_j M[l][j] a[j]
 * with qubit q = index bit q and qubits[0] the most significant local bit
 * (the Kronecker order of Eq. 1).  The sets are disjoint, so the outer loop
 * over s runs in parallel without changing any result: each output is the
 * same fixed-order FP64 sum whatever the thread count.  Build with
 * -ffp-contract=off so no fused multiply-add changes the rounding.
 *
 * Layout: psi and m are interleaved complex128 (re, im doubles), m is
 * 2^k x 2^k row-major.  1 <= k <= 10, distinct qubits < n <= 40.
 * Returns 0 on success, -1 on an argument error (nothing is written).
 */
#include <stdint.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAX_K 10

int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

int or_apply_gate(double* psi, int n, const int* qubits, int k, const double* m) {
    if (!psi || !qubits || !m || n < 1 || n > 40 || k < 1 || k > OR_MAX_K || k > n) return -1;
    for (int i = 0; i < k; ++i) {
        if (qubits[i] < 0 || qubits[i] >= n) return -1;
        for (int j = 0; j < i; ++j)
            if (qubits[i] == qubits[j]) return -1;
    }
    /* target bits in ascending order, for building the first index of a set */
    int sorted[OR_MAX_K];
    for (int i = 0; i < k; ++i) sorted[i] = qubits[i];
    for (int i = 1; i < k; ++i)
        for (int j = i; j > 0 && sorted[j - 1] > sorted[j]; --j) {
            int t = sorted[j];
            sorted[j] = sorted[j - 1];
            sorted[j - 1] = t;
        }
    const int64_t dim = (int64_t)1 << k;
    /* offset of local index l: bit (k-1-i) of l is qubit qubits[i] */
    int64_t* off = (int64_t*)malloc((size_t)dim * sizeof(int64_t));
    if (!off) return -1;
    for (int64_t l = 0; l < dim; ++l) {
        int64_t o = 0;
        for (int i = 0; i < k; ++i)
            if ((l >> (k - 1 - i)) & 1) o |= (int64_t)1 << qubits[i];
        off[l] = o;
    }
    const int64_t nsets = (int64_t)1 << (n - k);
    int failed = 0;
#pragma omp parallel
    {
        double* a = (double*)malloc((size_t)(2 * dim) * sizeof(double));
        if (!a) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(static)
        for (int64_t s = 0; s < nsets; ++s) {
            if (!a) continue;
            /* first index of set s: zero bits inserted at the targets */
            int64_t base = s;
            for (int i = 0; i < k; ++i) {
                const int b = sorted[i];
                const int64_t low = base & (((int64_t)1 << b) - 1);
                base = ((base >> b) << (b + 1)) | low;
            }
            for (int64_t l = 0; l < dim; ++l) {
                a[2 * l] = psi[2 * (base | off[l])];
                a[2 * l + 1] = psi[2 * (base | off[l]) + 1];
            }
            for (int64_t r = 0; r < dim; ++r) {
                double re = 0.0, im = 0.0;
                const double* row = m + 2 * r * dim;
                for (int64_t j = 0; j < dim; ++j) {
                    re += row[2 * j] * a[2 * j] - row[2 * j + 1] * a[2 * j + 1];
                    im += row[2 * j] * a[2 * j + 1] + row[2 * j + 1] * a[2 * j];
                }
                psi[2 * (base | off[r])] = re;
                psi[2 * (base | off[r]) + 1] = im;
            }
        }
        free(a);
    }
    free(off);
    return failed ? -1 : 0;
}
