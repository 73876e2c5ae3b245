/*
 * Plain complex128 state-vector oracle.  TEST INFRASTRUCTURE ONLY: the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark call it;
 * the product library never links, loads or runs it.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * What it computes is the plain definition of the method:
 *   - exact state-vector simulation (paper Sec. 1 and Sec. 4: both backends
 *     are noiseless state-vector simulators): psi = U_L ... U_1 |ref>, every
 *     gate applied as its explicit 2x2 (or controlled) matrix over index pairs;
 *   - direct expectation values of a Pauli sum, H = sum_i c_i P_i (Sec. 4.1,
 *     the paragraph casting Eq. 2 as generic terms P_i weighed by c_i):
 *     E = sum_i c_i <psi| P_i psi>, where P_i psi is built by applying the
 *     single-qubit Pauli matrices of the string one qubit at a time;
 *   - Eq. 1: <H>(theta) = <0| U^dag(theta) H U(theta) |0>, with |0> replaced
 *     by a reference basis state per instance.
 *
 * Readings where the paper is silent (qubit order, rotation convention) are:
 * qubit q = bit q of the basis index; R_P(a) = exp(-i a P / 2)
 * = cos(a/2) I - i sin(a/2) P.
 *
 * Parallelism: OpenMP over independent circuits only, mirroring the paper's
 * embarrassingly parallel execution model (Sec. 3); nothing inside one
 * circuit is vectorised, blocked or fused.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "sv_oracle.h"

typedef double complex cplx;

/* Gate codes: position in workloads.GATE_OPS. */
enum { G_RX = 0, G_RY, G_RZ, G_CNOT, G_X, G_H, G_CZ, G_ENC_RY_ASIN, G_ENC_RZ_ACOS_SQ };

/* The three Pauli matrices, written out. */
static void pauli_matrix(int letter, cplx m[2][2]) {
    m[0][0] = m[0][1] = m[1][0] = m[1][1] = 0.0;
    switch (letter) {
    case 1: /* X */
        m[0][1] = 1.0; m[1][0] = 1.0; break;
    case 2: /* Y */
        m[0][1] = -I; m[1][0] = I; break;
    case 3: /* Z */
        m[0][0] = 1.0; m[1][1] = -1.0; break;
    default: /* identity */
        m[0][0] = 1.0; m[1][1] = 1.0; break;
    }
}

/* R_P(a) = cos(a/2) I - i sin(a/2) P, for P = X (1), Y (2), Z (3). */
static void rotation_matrix(int letter, double a, cplx m[2][2]) {
    cplx p[2][2];
    pauli_matrix(letter, p);
    double c = cos(a / 2.0), s = sin(a / 2.0);
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 2; ++k)
            m[r][k] = (r == k ? c : 0.0) - I * s * p[r][k];
}

/* psi <- (m acting on qubit q) psi: every index pair differing only in bit q. */
static void apply_1q(cplx *psi, int n, int q, cplx m[2][2]) {
    long long dim = 1LL << n, bit = 1LL << q;
    for (long long j = 0; j < dim; ++j) {
        if (j & bit) continue;
        cplx a = psi[j], b = psi[j | bit];
        psi[j] = m[0][0] * a + m[0][1] * b;
        psi[j | bit] = m[1][0] * a + m[1][1] * b;
    }
}

/* CNOT: flips target bit t of every basis index whose control bit c is 1. */
static void apply_cnot(cplx *psi, int n, int c, int t) {
    long long dim = 1LL << n, cb = 1LL << c, tb = 1LL << t;
    for (long long j = 0; j < dim; ++j) {
        if ((j & cb) && !(j & tb)) {
            cplx tmp = psi[j];
            psi[j] = psi[j | tb];
            psi[j | tb] = tmp;
        }
    }
}

/* CZ: phase -1 on every basis index with both bits set. */
static void apply_cz(cplx *psi, int n, int a, int b) {
    long long dim = 1LL << n;
    for (long long j = 0; j < dim; ++j)
        if (((j >> a) & 1) && ((j >> b) & 1)) psi[j] = -psi[j];
}

static int apply_gate(cplx *psi, int n, int op, int target, int control, double angle,
                      const double *x) {
    cplx m[2][2];
    if (target < 0 || target >= n) return ORC_ERR_ARG;
    switch (op) {
    case G_RX: rotation_matrix(1, angle, m); apply_1q(psi, n, target, m); break;
    case G_RY: rotation_matrix(2, angle, m); apply_1q(psi, n, target, m); break;
    case G_RZ: rotation_matrix(3, angle, m); apply_1q(psi, n, target, m); break;
    case G_X: pauli_matrix(1, m); apply_1q(psi, n, target, m); break;
    case G_H: {
        /* H = (X + Z) / sqrt(2) */
        cplx px[2][2], pz[2][2];
        pauli_matrix(1, px); pauli_matrix(3, pz);
        for (int r = 0; r < 2; ++r)
            for (int k = 0; k < 2; ++k) m[r][k] = (px[r][k] + pz[r][k]) / sqrt(2.0);
        apply_1q(psi, n, target, m);
        break;
    }
    case G_CNOT:
        if (control < 0 || control >= n || control == target) return ORC_ERR_ARG;
        apply_cnot(psi, n, control, target);
        break;
    case G_CZ:
        if (control < 0 || control >= n || control == target) return ORC_ERR_ARG;
        apply_cz(psi, n, control, target);
        break;
    case G_ENC_RY_ASIN:
        if (!x) return ORC_ERR_ARG;
        rotation_matrix(2, asin(x[0]), m); apply_1q(psi, n, target, m); break;
    case G_ENC_RZ_ACOS_SQ:
        if (!x) return ORC_ERR_ARG;
        rotation_matrix(3, acos(x[0] * x[0]), m); apply_1q(psi, n, target, m); break;
    default:
        return ORC_ERR_ARG;
    }
    return ORC_OK;
}

static int run_circuit(const orc_circuit *c, const double *theta, int shift_param,
                       double shift, long long ref, const double *inputs, cplx *psi) {
    long long dim = 1LL << c->n_qubits;
    if (ref < 0 || ref >= dim) return ORC_ERR_ARG;
    for (long long j = 0; j < dim; ++j) psi[j] = 0.0;
    psi[ref] = 1.0;
    for (int g = 0; g < c->n_gates; ++g) {
        int op = c->op[g], p = c->param[g];
        double angle = c->angle[g];
        const double *x = NULL;
        if (op == G_ENC_RY_ASIN || op == G_ENC_RZ_ACOS_SQ) {
            if (!inputs || p < 0 || p >= c->input_dim) return ORC_ERR_ARG;
            x = inputs + p;
        } else if ((op == G_RX || op == G_RY || op == G_RZ) && p >= 0) {
            if (p >= c->n_params) return ORC_ERR_ARG;
            angle = theta[p] + (p == shift_param ? shift : 0.0);
        }
        int st = apply_gate(psi, c->n_qubits, op, c->target[g], c->control[g], angle, x);
        if (st != ORC_OK) return st;
    }
    return ORC_OK;
}

/* sum_t c_t <psi| P_t psi>, with P_t psi built one single-qubit Pauli at a time. */
static void expect(const cplx *psi, int n, int n_terms, const signed char *letters,
                   const double *coeffs, cplx *work, double *out_re, double *out_im) {
    long long dim = 1LL << n;
    cplx total = 0.0;
    for (int t = 0; t < n_terms; ++t) {
        memcpy(work, psi, sizeof(cplx) * (size_t)dim);
        for (int q = 0; q < n; ++q) {
            int l = letters[(size_t)t * n + q];
            if (l == 0) continue;
            cplx m[2][2];
            pauli_matrix(l, m);
            apply_1q(work, n, q, m);
        }
        cplx ip = 0.0;
        for (long long j = 0; j < dim; ++j) ip += conj(psi[j]) * work[j];
        total += coeffs[t] * ip;
    }
    *out_re = creal(total);
    *out_im = cimag(total);
}

int orc_state(const orc_circuit *c, const double *theta, int shift_param, double shift,
              long long ref, const double *inputs, double *psi_out) {
    if (!c || c->n_qubits < 1 || c->n_qubits > 30) return ORC_ERR_ARG;
    return run_circuit(c, theta, shift_param, shift, ref, inputs, (cplx *)psi_out);
}

int orc_expect_state(const double *psi, int n, int n_terms, const signed char *letters,
                     const double *coeffs, double *out_re, double *out_im) {
    long long dim = 1LL << n;
    cplx *work = malloc(sizeof(cplx) * (size_t)dim);
    if (!work) return ORC_ERR_OOM;
    expect((const cplx *)psi, n, n_terms, letters, coeffs, work, out_re, out_im);
    free(work);
    return ORC_OK;
}

int orc_energies(const orc_circuit *c, const double *theta, int n_terms,
                 const signed char *letters, const double *coeffs, int n_slots,
                 const long long *slot_ref, const double *slot_inputs,
                 const int *slot_shift_param, const double *slot_shift,
                 double *out_re, double *out_im, int n_threads) {
    if (!c || c->n_qubits < 1 || c->n_qubits > 30 || n_slots < 0) return ORC_ERR_ARG;
    long long dim = 1LL << c->n_qubits;
    int status = ORC_OK;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
#pragma omp parallel
    {
        cplx *psi = malloc(sizeof(cplx) * (size_t)dim);
        cplx *work = malloc(sizeof(cplx) * (size_t)dim);
        if (!psi || !work) {
#pragma omp atomic write
            status = ORC_ERR_OOM;
        }
#pragma omp for schedule(dynamic, 1)
        for (int s = 0; s < n_slots; ++s) {
            if (!psi || !work) continue;
            const double *x = slot_inputs ? slot_inputs + (size_t)s * c->input_dim : NULL;
            int st = run_circuit(c, theta, slot_shift_param ? slot_shift_param[s] : -1,
                                 slot_shift ? slot_shift[s] : 0.0, slot_ref[s], x, psi);
            if (st != ORC_OK) {
#pragma omp atomic write
                status = st;
                continue;
            }
            expect(psi, c->n_qubits, n_terms, letters, coeffs, work, &out_re[s], &out_im[s]);
        }
        free(psi);
        free(work);
    }
    return status;
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
