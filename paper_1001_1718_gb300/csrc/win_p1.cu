// Register-window forward kernels, part 1 of win.cu (see its header).
#define WIN_PART 1
#include "win.cu"
