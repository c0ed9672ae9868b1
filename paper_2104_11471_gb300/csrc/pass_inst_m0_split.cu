// Pass kernels for mode 0, split precision, every supported length.
#include "pass_inst.cuh"
TCFFT_PASS_UNIT(0, true, pass_fn_m0_split)
