// Register-window forward kernels, part 3 of win.cu (see its header).
#define WIN_PART 3
#include "win.cu"
