// rtt_simt_f64.cu -- FP64 instantiation of the SIMT kernels (rtt_simt.cuh).
// Reproduces the oracle's canonical fma order; compiled with -fmad=false.
#include "rtt_simt.cuh"

RTT_DEFINE_SIMT(double, f64)
