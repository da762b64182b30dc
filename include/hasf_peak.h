/*
 * hasf_peak.h -- measurement helper of the benchmark (libhasf_peak.so), not
 * part of the filter's ABI and without a counterpart in the paper.
 *
 * The HASF kernels are integer-issue bound: their work is 32-bit logic
 * (LOP3), funnel shifts (SHF), additions (IADD3) and warp shuffles (SHFL).
 * hasf_peak_int measures how many lane-operations per second one of these
 * classes sustains on the whole GPU, so that the benchmark's "alu" roofline
 * divides by a measured rate rather than a nominal one.
 */
#ifndef HASF_PEAK_H_
#define HASF_PEAK_H_

#ifdef __cplusplus
extern "C" {
#endif

enum {
    HASF_PEAK_LOP3 = 0,   /* three-input logic, a = (a & b) ^ c            */
    HASF_PEAK_SHF = 1,    /* funnel shift, a = funnelshift_r(a, b, s)      */
    HASF_PEAK_IADD3 = 2,  /* three-input add, a = a + a' + c (a' another chain) */
    HASF_PEAK_SHFL = 3    /* warp shuffle, a = shfl_xor(a, m)              */
};

/* Run the probe of instruction class `kind` on CUDA device `device` (made
 * current) and store its rate in *lane_ops_per_s (warp instructions x 32 per
 * second) and the timed launch's duration in *ms (may be NULL).  Allocates
 * and frees its own small device buffer; synchronous.
 * Returns 0, 1 for a bad argument, 2 for a CUDA error. */
int hasf_peak_int(int kind, int device, double *lane_ops_per_s, float *ms);

#ifdef __cplusplus
}
#endif

#endif /* HASF_PEAK_H_ */
