/*
 * ht.h -- C ABI of the GB300 many-path polynomial homotopy tracker.
 *
 * The operations follow Verschelde & Yu, "Tracking Many Solution Paths of a
 * Polynomial Homotopy on a Graphics Processing Unit" (2015):
 *   - the homotopy gamma (1 - t) g(x) + t f(x) = 0 of Eq. (eqlinhom), Section 1;
 *   - evaluation and differentiation of all monomials at many points with the
 *     reverse mode of Table tabmoneval, Section 3;
 *   - the predictor-corrector loop over many paths, Section 2, with Newton's
 *     method solving each linear system in the least squares sense by modified
 *     Gram-Schmidt (Section 1), the status codes and the scan compaction of
 *     Table tabjobidx.
 *
 * Conventions shared by every entry point:
 *   - Every function returns an int: HT_OK (0) on success, a negative HT_E*
 *     code on failure; ht_last_error() then holds a message for the calling
 *     thread.  No C++ exception crosses this interface.
 *   - Precision is given as the number of limbs L per real number: 1 complex
 *     double, 2 complex double double, 4 complex quad double (Section 1,
 *     Section 4.1).  A real number is the unevaluated sum of its L doubles,
 *     limb 0 the leading one.
 *   - Batches of points are stored "vertically" (Section 3, Table tabtranspose):
 *     a quantity with `count` complex entries over `n` points is the array
 *     [count][2][L][n] of doubles -- entry, real/imaginary part, limb, point --
 *     so all points' values of one limb of one entry are contiguous.
 *   - Buffers named "device" are caller-owned CUDA device memory on the current
 *     device, 8-byte aligned; the library neither frees nor keeps them.  Calls
 *     taking a `stream` enqueue work on that cudaStream_t (NULL = legacy default
 *     stream) and return before it finishes unless stated otherwise.
 *   - Invalid arguments are rejected with HT_EINVAL before any launch.
 *
 * Accuracy contract of the arithmetic: every computed value differs from the
 * exact value of the same formula by at most a small multiple of 2^(-53 L)
 * times the sum of the moduli of the terms that make it up.
 */
#ifndef HT_H
#define HT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { HT_D = 1, HT_DD = 2, HT_QD = 4 };

enum {
  HT_OK = 0,
  HT_EINVAL = -1,       /* invalid argument */
  HT_ENOMEM = -2,       /* device or host allocation failed */
  HT_ECUDA = -3,        /* a CUDA call failed (message in ht_last_error) */
  HT_ETIMEOUT = -4,     /* a bounded device-side wait expired */
  HT_EUNSUPPORTED = -5  /* valid but not supported (e.g. too many variables) */
};

/* Opaque, library-owned polynomial system ("instructions" of Table tabmemory:
 * the monomial supports (idx) and coefficients (cff), shared by all paths). */
typedef struct ht_system ht_system;

/* Message of the last failing call on this thread ("" if none). */
const char* ht_last_error(void);

/*
 * ht_create_system -- copy a polynomial system to the device (Table tabmemory).
 *   n_vars   number of variables, 1..255
 *   n_polys  number of polynomials, >= 1
 *   n_terms  host [n_polys]: monomials in each polynomial, each >= 1
 *   exps     host [M][n_vars] (M = sum of n_terms): exponents, 0..127,
 *            polynomial 0's monomials first
 *   coef     host [M][2][limbs]: complex coefficients (re limbs, im limbs)
 *   limbs    HT_D, HT_DD or HT_QD: the precision evaluations use
 *   out      receives the handle; release it with ht_destroy_system
 * Uses the current CUDA device.  Errors: HT_EINVAL for bad shapes or values,
 * HT_EUNSUPPORTED for a monomial with more than 64 variables, HT_ENOMEM,
 * HT_ECUDA.
 */
int ht_create_system(int n_vars, int n_polys, const int32_t* n_terms, const int8_t* exps,
                     const double* coef, int limbs, ht_system** out);

/* Release a system (NULL is accepted).  Waits for the device to finish. */
int ht_destroy_system(ht_system* sys);

/* Shape of a system: any output pointer may be NULL. */
int ht_system_info(const ht_system* sys, int* n_vars, int* n_polys, int* limbs, int64_t* n_monomials);

/*
 * ht_eval_diff -- evaluate every polynomial and its Jacobian at n_pts points
 * (Section 3, Table tabcpugpu: coefficient, monomial value and derivatives by
 * the reverse mode of Table tabmoneval, sums into the polynomial and the
 * Jacobian, here fused in one kernel).
 *   x    device [n_vars][2][L][n_pts]   points
 *   val  device [n_polys][2][L][n_pts]  receives f_j(x_p)
 *   jac  device [n_polys][n_vars][2][L][n_pts] receives df_j/dx_i (x_p)
 * L is the system's precision.  n_pts == 0 is a no-op.  x must not overlap val
 * or jac.  Asynchronous on `stream`.
 */
int ht_eval_diff(const ht_system* sys, int64_t n_pts, const double* x, double* val, double* jac,
                 void* stream);

/*
 * ht_eval_diff_host -- ht_eval_diff on HOST buffers of the same layouts: copies
 * x to the device, evaluates, copies val and jac back, and returns when the
 * results are in host memory.  Uses a device workspace owned by the system
 * (grown on demand, freed with the system).  Pinned host memory gives the
 * fastest copies; pageable memory works.
 */
int ht_eval_diff_host(ht_system* sys, int64_t n_pts, const double* x_host, double* val_host,
                      double* jac_host, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HT_H */
