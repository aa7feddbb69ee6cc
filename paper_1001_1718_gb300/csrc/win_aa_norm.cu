// Antialiased fused pre-process kernels, part 1 of win_aa.cu (see its header).
#define WIN_AA_PART 1
#include "win_aa.cu"
