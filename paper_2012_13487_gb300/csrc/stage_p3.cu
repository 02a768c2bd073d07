// Fused LSRK stage kernel instantiated for polynomial degree 3.
#define FEDBM_P 3
#define FEDBM_STAGE_ENTRY_NAME stage_entry_p3
#include "stage_impl.cuh"
