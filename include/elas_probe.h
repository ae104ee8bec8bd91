/*
 * elas_probe -- measurement utility of libelas_gb300 (the paper has no
 * counterpart).  Used by the benchmark to measure the integer-ALU ceiling of
 * the 16-byte SAD that the support and dense matchers are built on.
 */
#ifndef ELAS_PROBE_H
#define ELAS_PROBE_H
#include <stdint.h>
#include "elas_gb300.h"
#ifdef __cplusplus
extern "C" {
#endif
/*
 * Runs blocks x threads threads, each evaluating iters * 8 SAD16 (16 byte
 * absolute differences summed) on register-resident data; time it with CUDA
 * events on `stream`.  variant 0: __vabsdiffu4 + __dp4a (the kernels'
 * sequence); 1: __vsadu4; 2: PTX vabsdiff4 with accumulate.  scratch: device,
 * blocks*threads uint32 (written only in a practically impossible branch).
 */
elas_status elas_probe_sad16(int32_t variant, int32_t blocks, int32_t threads, int32_t iters,
                             uint32_t *scratch, elas_stream stream);
#ifdef __cplusplus
}
#endif
#endif
