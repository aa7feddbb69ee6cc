// Fused pre-process kernels, the exact-x2 part of win_norm.cu (see its header).
#define WIN_NORM_PART 1
#include "win_norm.cu"
