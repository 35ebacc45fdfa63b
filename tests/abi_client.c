/*
 * A plain C client of the checker's C-ABI (no CUDA headers, no C++): builds
 * Listing 1's race in host memory - thread 0 of block 0 writes word 0 while
 * thread 0 of block 1 reads it, with a __syncthreads between that cannot
 * order two blocks (Sec. II-B) - checks it through hr_check_trace_host and
 * prints the reports.  Built and run by tests/test_gpu_abi_client.py.
 */
#include <stdio.h>
#include <string.h>

#include "hirace.h"

static hr_record rec(uint32_t word, uint32_t tid, uint16_t bc, uint8_t op)
{
    hr_record r;
    memset(&r, 0, sizeof r);
    r.word = word;
    r.tid = tid;
    r.bc = bc;
    r.op = op;
    return r;
}

int main(void)
{
    /* block_dim 2: tids 0,1 are block 0, tids 2,3 block 1; records in wave order */
    hr_record trace[8];
    int n = 0;
    trace[n++] = rec(0, 0, 0, HR_W);            /* block 0 writes word 0 in epoch 0 */
    trace[n++] = rec(1, 2, 0, HR_R);            /* block 1 reads word 1: no conflict */
    for (uint32_t t = 0; t < 4; ++t) trace[n++] = rec(0, t, 1, HR_SYNCTHREADS);
    trace[n++] = rec(0, 2, 1, HR_R);            /* block 1 reads word 0 after its barrier */
    trace[n++] = rec(1, 1, 1, HR_R);            /* block 0 reads word 1: reads never race */

    hr_region_desc d;
    memset(&d, 0, sizeof d);
    d.n_words = 4;
    d.block_dim = 2;
    d.warp_size = 32;
    hr_ctx* ctx = NULL;
    hr_status st = hr_init(&ctx, &d, 1, 64, NULL);
    if (st != HR_OK) {
        printf("hr_init: %s\n", hr_status_str(st));
        return 1;
    }
    st = hr_check_trace_host(ctx, 0, trace, (uint64_t)n, 0, NULL);
    if (st != HR_OK) {
        printf("hr_check_trace_host: %s\n", hr_status_str(st));
        return 1;
    }
    hr_race races[8];
    uint64_t total = 0;
    uint32_t flags = 0;
    st = hr_report(ctx, 0, races, 8, &total, &flags);
    printf("status %s races %llu flags %u\n", hr_status_str(st), (unsigned long long)total, flags);
    for (uint64_t i = 0; i < total && i < 8; ++i)
        printf("race word %u kernel %u epoch %u tid %u op %u prior %s\n", races[i].word, races[i].kernel,
               races[i].epoch, races[i].tid, races[i].op, hr_fsm_state_name(races[i].prior));
    hr_destroy(ctx);
    return st == HR_OK ? 0 : 1;
}
