// Pass kernels for mode 0, plain precision, every supported length.
#include "pass_inst.cuh"
TCFFT_PASS_UNIT(0, false, pass_fn_m0_plain)
