// Adjoint kernels of one RK stage (placeholder translation unit).
#include "dg_internal.h"
