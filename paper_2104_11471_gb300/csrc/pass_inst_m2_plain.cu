// Pass kernels for mode 2, plain precision, every supported length.
#include "pass_inst.cuh"
TCFFT_PASS_UNIT(2, false, pass_fn_m2_plain)
