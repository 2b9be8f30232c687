/*
 * Oracle (test infrastructure only): particle codes, the stable sort and
 * the physical-block set of the rebuild-mapping phase.
 *
 * Sec. 4: the particle code interleaves the three integer indices; the high
 * bits are the block code, the low bits the cell code.  Sec. 4.2.2: the
 * histogram sort keys each particle by its block's index followed by its
 * cell code; with the block index equal to the rank of the block's Morton code, the
 * sort order is the order of (Morton(block) << 6 | Morton(cell)).
 * Sec. 4.2.1: particle blocks are shifted by -dx/2 (base = floor(x/dx - 1/2))
 * and the physical blocks are the gblocks with their 3x3x3 neighbours.
 *
 * The key is an integer decided from FP32 positions, so it is computed here
 * in FP32 arithmetic, the precision the GPU path decides it in.  Morton bit
 * order: x in the lowest bit of each triple, then y, then z.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static uint32_t interleave(uint32_t bx, uint32_t by, uint32_t bz, int bits)
{
    uint32_t code = 0;
    for (int i = 0; i < bits; ++i) {
        code |= ((bx >> i) & 1u) << (3 * i);
        code |= ((by >> i) & 1u) << (3 * i + 1);
        code |= ((bz >> i) & 1u) << (3 * i + 2);
    }
    return code;
}

static void deinterleave(uint32_t code, int bits, int32_t c[3])
{
    c[0] = c[1] = c[2] = 0;
    for (int i = 0; i < bits; ++i)
        for (int a = 0; a < 3; ++a)
            c[a] |= (int32_t)(((code >> (3 * i + a)) & 1u) << i);
}

int orc_particle_keys(int64_t n, const float* x, float inv_dx, int32_t L, uint32_t* keys)
{
    int status = ORC_OK;
    for (int64_t p = 0; p < n; ++p) {
        int32_t base[3];
        for (int a = 0; a < 3; ++a) {
            volatile float X = x[3 * p + a] * inv_dx;   /* FP32 product */
            volatile float Y = X - 0.5f;                /* FP32 difference */
            base[a] = (int32_t)floorf(Y);
        }
        uint32_t blk[3], cel[3];
        int bad = 0;
        for (int a = 0; a < 3; ++a) {
            if (base[a] < 0 || (base[a] >> 2) >= (1 << L))
                bad = 1;
            blk[a] = (uint32_t)(base[a] >> 2);
            cel[a] = (uint32_t)(base[a] & 3);
        }
        if (bad) {
            status = ORC_EDOMAIN;
            keys[p] = 0xffffffffu;
            continue;
        }
        keys[p] = (interleave(blk[0], blk[1], blk[2], L) << 6) | interleave(cel[0], cel[1], cel[2], 2);
    }
    return status;
}

/* bottom-up merge sort of indices by key; merge takes from the left run
 * on ties, so equal keys keep their original order */
void orc_stable_sort(int64_t n, const uint32_t* keys, int32_t* perm)
{
    int32_t* tmp = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    for (int64_t i = 0; i < n; ++i)
        perm[i] = (int32_t)i;
    int32_t* src = perm;
    int32_t* dst = tmp;
    for (int64_t width = 1; width < n; width *= 2) {
        for (int64_t lo = 0; lo < n; lo += 2 * width) {
            int64_t mid = lo + width < n ? lo + width : n;
            int64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
            int64_t i = lo, j = mid, k = lo;
            while (i < mid && j < hi)
                dst[k++] = keys[src[j]] < keys[src[i]] ? src[j++] : src[i++];
            while (i < mid)
                dst[k++] = src[i++];
            while (j < hi)
                dst[k++] = src[j++];
        }
        int32_t* t = src;
        src = dst;
        dst = t;
    }
    if (src != perm)
        memcpy(perm, src, (size_t)n * sizeof(int32_t));
    free(tmp);
}

int64_t orc_pblocks(int64_t n, const uint32_t* keys, int32_t L, int32_t* out)
{
    int64_t slots = (int64_t)1 << (3 * L);
    unsigned char* mark = (unsigned char*)calloc((size_t)slots, 1);
    int32_t side = 1 << L;
    for (int64_t p = 0; p < n; ++p) {
        if (keys[p] == 0xffffffffu)
            continue;
        int32_t b[3];
        deinterleave(keys[p] >> 6, L, b);
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int32_t c[3] = {b[0] + dx, b[1] + dy, b[2] + dz};
                    if (c[0] < 0 || c[1] < 0 || c[2] < 0 || c[0] >= side || c[1] >= side || c[2] >= side)
                        continue;
                    mark[interleave((uint32_t)c[0], (uint32_t)c[1], (uint32_t)c[2], L)] = 1;
                }
    }
    int64_t count = 0;
    for (int64_t s = 0; s < slots; ++s)
        if (mark[s]) {
            if (out)
                out[count] = (int32_t)s;
            ++count;
        }
    free(mark);
    return count;
}
