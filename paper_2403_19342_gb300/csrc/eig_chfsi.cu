// Level-1 local eigensolver for large elements (placeholder until the
// subspace solver lands).
#include "msmg_internal.cuh"
namespace msmg {
int launch_level1_chfsi(msmg_ctx* c, cudaStream_t s) { (void)c; (void)s; return MSMG_ERR_UNSUPPORTED; }
}
