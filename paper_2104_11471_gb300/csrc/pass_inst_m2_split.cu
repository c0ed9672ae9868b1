// Pass kernels for mode 2, split precision, every supported length.
#include "pass_inst.cuh"
TCFFT_PASS_UNIT(2, true, pass_fn_m2_split)
