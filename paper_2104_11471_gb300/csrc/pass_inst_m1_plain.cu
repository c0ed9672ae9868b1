// Pass kernels for mode 1, plain precision, every supported length.
#include "pass_inst.cuh"
TCFFT_PASS_UNIT(1, false, pass_fn_m1_plain)
