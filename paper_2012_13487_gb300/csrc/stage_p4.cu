// Fused LSRK stage kernel instantiated for polynomial degree 4.
#define FEDBM_P 4
#define FEDBM_STAGE_ENTRY_NAME stage_entry_p4
#include "stage_impl.cuh"
