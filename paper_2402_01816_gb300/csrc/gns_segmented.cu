// gns_segmented.cu -- batched segmented sort (placeholder entry points).
#include "gns_internal.h"

extern "C" {

int gns_segmented_sort(int64_t* keys, uint32_t* payload, const int64_t* offsets, int64_t nseg,
                       gns_stream_t stream)
{
    (void)keys; (void)payload; (void)offsets; (void)nseg; (void)stream;
    return GNS_ERR_UNSUPPORTED;
}

int gns_segmented_sort_ex(void* keys, int key_type, uint32_t* payload, const int64_t* offsets, int64_t nseg,
                          int64_t total_n, int order, gns_stream_t stream)
{
    (void)keys; (void)key_type; (void)payload; (void)offsets; (void)nseg; (void)total_n; (void)order;
    (void)stream;
    return GNS_ERR_UNSUPPORTED;
}

}  // extern "C"
