// ecc_tune.cu -- tile-parameter selection (autotuner).
#include "ecc_plan.h"

void ecc_plan_s::autotune() {}
