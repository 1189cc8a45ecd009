/*
 * qt_oracle.c -- plain FP64 CPU oracle for state-vector circuit simulation.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file; only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no header, table or helper with
 * the CUDA path: gate matrices are written out here from their definitions,
 * and the amplitude updates are the textbook loops, with no blocking, fusion
 * or reordering.
 *
 * What it computes (qTask, Section II-A): an n-qubit state is 2^n complex
 * amplitudes alpha_b, b = q_{n-1}...q_1 q_0 in binary with q_0 the least
 * significant bit, and sum_b |alpha_b|^2 = 1.  A circuit is an ordered list
 * of levels ("nets", Section III-B); the output state is the ordered product
 * of the level unitaries applied to |0...0>.  Gates inside one level act on
 * disjoint qubits, so they commute and are applied here one after another.
 *
 * Gate conventions (the paper prints only X, H and CX, Section II-A; it
 * names the rest of its gate table, Table 1, and the composites CZ, CCX and
 * SWAP, Section III-A):
 *   X = [[0,1],[1,0]], H = [[1,1],[1,-1]]/sqrt2, Y = [[0,-i],[i,0]],
 *   Z = diag(1,-1), S = diag(1,i), SDG = diag(1,-i), T = diag(1,e^{i pi/4}),
 *   TDG = diag(1,e^{-i pi/4}),
 *   RX(t) = [[c,-is],[-is,c]], RY(t) = [[c,-s],[s,c]],
 *   RZ(t) = diag(e^{-it/2}, e^{it/2}), with c = cos(t/2), s = sin(t/2),
 *   U3(t,p,l) = [[c, -e^{il} s], [e^{ip} s, e^{i(p+l)} c]],
 *   P(l) = diag(1, e^{il})  (the target of the controlled phase CP),
 *   CNOT = controlled X, CZ = controlled Z, CCX = X with two controls,
 *   SWAP = the 4x4 permutation exchanging the two target bits.
 * A controlled gate applies its base matrix to exactly those amplitudes whose
 * control bits are all 1 (the CX matrix of Section II-A).
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC qt_oracle.c -o libqt_oracle.so -lm
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* ---------------------------------------------------------------- gates -- */

/* Base matrix of a named gate, written row-major into U (dim x dim, dim = 2
 * for one-target gates, 4 for SWAP).  Returns dim, or 0 for an unknown name.
 * params holds up to three angles (theta, phi, lambda).                     */
int orc_base_matrix(const char* name, const double* params, double* U_ri)
{
    cplx U[16];
    int dim = 2;
    const double r2 = 1.0 / sqrt(2.0);
    double t = params ? params[0] : 0.0;
    double c = cos(t / 2.0), s = sin(t / 2.0);
    for (int k = 0; k < 16; ++k) U[k] = 0.0;
    if (!strcmp(name, "x") || !strcmp(name, "cnot") || !strcmp(name, "ccx")) {
        U[0] = 0; U[1] = 1; U[2] = 1; U[3] = 0;
    } else if (!strcmp(name, "h")) {
        U[0] = r2; U[1] = r2; U[2] = r2; U[3] = -r2;
    } else if (!strcmp(name, "y")) {
        U[0] = 0; U[1] = -I; U[2] = I; U[3] = 0;
    } else if (!strcmp(name, "z") || !strcmp(name, "cz")) {
        U[0] = 1; U[3] = -1;
    } else if (!strcmp(name, "s")) {
        U[0] = 1; U[3] = I;
    } else if (!strcmp(name, "sdg")) {
        U[0] = 1; U[3] = -I;
    } else if (!strcmp(name, "t")) {
        U[0] = 1; U[3] = cexp(I * M_PI / 4.0);
    } else if (!strcmp(name, "tdg")) {
        U[0] = 1; U[3] = cexp(-I * M_PI / 4.0);
    } else if (!strcmp(name, "rx")) {
        U[0] = c; U[1] = -I * s; U[2] = -I * s; U[3] = c;
    } else if (!strcmp(name, "ry")) {
        U[0] = c; U[1] = -s; U[2] = s; U[3] = c;
    } else if (!strcmp(name, "rz")) {
        U[0] = cexp(-I * t / 2.0); U[3] = cexp(I * t / 2.0);
    } else if (!strcmp(name, "u3")) {
        double p = params[1], l = params[2];
        U[0] = c; U[1] = -cexp(I * l) * s;
        U[2] = cexp(I * p) * s; U[3] = cexp(I * (p + l)) * c;
    } else if (!strcmp(name, "cp")) {
        U[0] = 1; U[3] = cexp(I * t);
    } else if (!strcmp(name, "swap")) {
        dim = 4;
        /* sub-index r = b_{t1} * 2 + b_{t0}; SWAP exchanges 01 and 10 */
        U[0 * 4 + 0] = 1; U[1 * 4 + 2] = 1; U[2 * 4 + 1] = 1; U[3 * 4 + 3] = 1;
    } else {
        return 0;
    }
    for (int k = 0; k < dim * dim; ++k) {
        U_ri[2 * k] = creal(U[k]);
        U_ri[2 * k + 1] = cimag(U[k]);
    }
    return dim;
}

/* ------------------------------------------------------- gate application */

/* Apply a one-target matrix U to target t, restricted to amplitudes whose
 * control bits (mask cmask) are all 1.  For every index i with bit t = 0,
 * the pair (a_i, a_j), j = i | 2^t, is replaced by U (a_i, a_j)^T.        */
static void apply_1t(int n, cplx* a, const cplx* U, int t, uint64_t cmask, int nthreads)
{
    const int64_t N = (int64_t)1 << n;
    const uint64_t tb = (uint64_t)1 << t;
    (void)nthreads;
#pragma omp parallel for schedule(static) num_threads(nthreads) if (nthreads > 1)
    for (int64_t i = 0; i < N; ++i) {
        if ((uint64_t)i & tb) continue;
        if (((uint64_t)i & cmask) != cmask) continue;
        int64_t j = i | (int64_t)tb;
        cplx x0 = a[i], x1 = a[j];
        a[i] = U[0] * x0 + U[1] * x1;
        a[j] = U[2] * x0 + U[3] * x1;
    }
}

/* Apply a two-target 4x4 matrix U to targets (t0, t1); the 4x4 sub-index of
 * an amplitude is r = 2*b_{t1} + b_{t0}.                                    */
static void apply_2t(int n, cplx* a, const cplx* U, int t0, int t1, uint64_t cmask, int nthreads)
{
    const int64_t N = (int64_t)1 << n;
    const uint64_t b0 = (uint64_t)1 << t0, b1 = (uint64_t)1 << t1;
    (void)nthreads;
#pragma omp parallel for schedule(static) num_threads(nthreads) if (nthreads > 1)
    for (int64_t i = 0; i < N; ++i) {
        if ((uint64_t)i & (b0 | b1)) continue;
        if (((uint64_t)i & cmask) != cmask) continue;
        int64_t idx[4] = { i, i | (int64_t)b0, i | (int64_t)b1, i | (int64_t)(b0 | b1) };
        cplx x[4], y[4];
        for (int r = 0; r < 4; ++r) x[r] = a[idx[r]];
        for (int r = 0; r < 4; ++r) {
            y[r] = 0;
            for (int k = 0; k < 4; ++k) y[r] += U[r * 4 + k] * x[k];
        }
        for (int r = 0; r < 4; ++r) a[idx[r]] = y[r];
    }
}

/* Apply one named gate to psi (2^n amplitudes, interleaved re/im doubles).
 * targets[0..ntarget-1], controls[0..ncontrol-1] are qubit numbers.
 * Returns 0 on success, -1 on a bad gate.                                   */
int orc_apply_gate(int n, double* psi, const char* name, int ntarget, const int* targets,
                   int ncontrol, const int* controls, const double* params, int nthreads)
{
    double Uri[32];
    cplx U[16];
    int dim = orc_base_matrix(name, params, Uri);
    if (dim == 0) return -1;
    if ((dim == 2 && ntarget != 1) || (dim == 4 && ntarget != 2)) return -1;
    for (int k = 0; k < dim * dim; ++k) U[k] = Uri[2 * k] + I * Uri[2 * k + 1];
    uint64_t cmask = 0, used = 0;
    for (int k = 0; k < ntarget; ++k) {
        if (targets[k] < 0 || targets[k] >= n || (used >> targets[k] & 1)) return -1;
        used |= (uint64_t)1 << targets[k];
    }
    for (int k = 0; k < ncontrol; ++k) {
        if (controls[k] < 0 || controls[k] >= n || (used >> controls[k] & 1)) return -1;
        used |= (uint64_t)1 << controls[k];
        cmask |= (uint64_t)1 << controls[k];
    }
    if (nthreads < 1) nthreads = 1;
    if (dim == 2)
        apply_1t(n, (cplx*)psi, U, targets[0], cmask, nthreads);
    else
        apply_2t(n, (cplx*)psi, U, targets[0], targets[1], cmask, nthreads);
    return 0;
}

/* Full simulation from |0...0> of a flat gate list given in application
 * order (levels already concatenated).  Per gate g: names[g]; ntarget[g]
 * targets in targets[2g..]; ncontrol[g] controls in controls[2g..]; three
 * angles in params[3g..].  psi_out receives 2^n interleaved amplitudes.    */
int orc_simulate(int n, int ngates, const char* const* names, const int* ntarget,
                 const int* targets, const int* ncontrol, const int* controls,
                 const double* params, double* psi_out, int nthreads)
{
    if (n < 1 || n > 34) return -1;
    const int64_t N = (int64_t)1 << n;
    memset(psi_out, 0, sizeof(double) * 2 * (size_t)N);
    psi_out[0] = 1.0;
    for (int g = 0; g < ngates; ++g) {
        int rc = orc_apply_gate(n, psi_out, names[g], ntarget[g], targets + 2 * g,
                                ncontrol[g], controls + 2 * g, params + 3 * g, nthreads);
        if (rc) return -(g + 2);
    }
    return 0;
}

/* sum_b |alpha_b|^2, accumulated in FP64 in index order (Section II-A).   */
double orc_norm(int n, const double* psi)
{
    const int64_t N = (int64_t)1 << n;
    double s = 0.0;
    for (int64_t i = 0; i < N; ++i) s += psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1];
    return s;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
