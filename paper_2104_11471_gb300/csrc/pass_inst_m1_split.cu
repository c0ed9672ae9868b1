// Pass kernels for mode 1, split precision, every supported length.
#include "pass_inst.cuh"
TCFFT_PASS_UNIT(1, true, pass_fn_m1_split)
