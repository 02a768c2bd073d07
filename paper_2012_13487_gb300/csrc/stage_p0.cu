// Fused LSRK stage kernel instantiated for polynomial degree 0.
#define FEDBM_P 0
#define FEDBM_STAGE_ENTRY_NAME stage_entry_p0
#include "stage_impl.cuh"
