/*
 * Plain complex128 state-vector oracle (test infrastructure only).
 * Amplitudes are interleaved (re, im) doubles, qubit q = bit q of the index.
 */
#ifndef SV_ORACLE_H
#define SV_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_OOM = 2 };

/* A circuit as parallel arrays; op codes are positions in workloads.GATE_OPS. */
typedef struct {
    int n_qubits;
    int n_gates;
    int n_params;
    int input_dim;
    const int *op;
    const int *target;
    const int *control;
    const int *param;
    const double *angle;
} orc_circuit;

/* Final state of one circuit from |ref>, with theta[shift_param] += shift. */
int orc_state(const orc_circuit *c, const double *theta, int shift_param, double shift,
              long long ref, const double *inputs, double *psi_out);

/* sum_t coeffs[t] <psi| P_t |psi> for Pauli rows letters[t*n + q] in {0:I,1:X,2:Y,3:Z}. */
int orc_expect_state(const double *psi, int n, int n_terms, const signed char *letters,
                     const double *coeffs, double *out_re, double *out_im);

/* Energies of many slots (reference, inputs row, shifted parameter, shift). */
int orc_energies(const orc_circuit *c, const double *theta, int n_terms,
                 const signed char *letters, const double *coeffs, int n_slots,
                 const long long *slot_ref, const double *slot_inputs,
                 const int *slot_shift_param, const double *slot_shift,
                 double *out_re, double *out_im, int n_threads);

int orc_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
