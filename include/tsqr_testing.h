/*
 * tsqr_testing.h -- entry points of libtsqr_gb300.so that run one internal
 * device step of the factorisation on caller-supplied inputs, so that the
 * test suite can check that step's arithmetic against the mathematics it
 * implements.  They are not needed to use the library.
 */
#ifndef TSQR_GB300_TESTING_H
#define TSQR_GB300_TESTING_H

#include <stdint.h>

#include "tsqr.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * tsqr_test_reflectors: the Householder reflector of the leaf and tree-node
 * kernels (H = I - tau u u^T with u = [1; t * scale], beta = -sign(alpha)
 * ||x||, x = [alpha; t], Section 4's normalisation) for `count` inputs,
 * each given as alpha[i] and the squared tail norm ssq[i] = ||t||^2.
 *   fast = 0: the reference form (IEEE sqrt and division);
 *   fast = 1: the short-latency form used on each column's serial step
 *             (FP32 seeds refined by one third-order correction), which falls
 *             back to the reference form outside its safe input range.
 *   alpha, ssq: device arrays of count doubles (read);
 *   out: device array of 3 * count doubles, out[3i..3i+2] = beta, tau,
 *        scale of input i (written).
 * Inputs whose tail must be rescanned (zero, tiny or huge ssq) take the
 * rescan result sqrt(ssq).  Asynchronous on `stream`; returns 0 or a
 * TSQR_ERR_* / -i code.
 */
int tsqr_test_reflectors(int64_t count, const double* alpha, const double* ssq, int32_t fast, double* out,
                         tsqr_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* TSQR_GB300_TESTING_H */
