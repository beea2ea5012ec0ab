/*
 * orc_rng.c -- oracle Philox4x32-10 (test infrastructure only).
 *
 * Philox4x32 as published by Salmon, Moraes, Dror and Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3" (SC'11): ten rounds, each multiplying words 0
 * and 2 by the two round multipliers, swapping halves and xoring with the
 * round key; the key is bumped by the two Weyl constants between rounds.
 *
 * Stream layout (one stream per photon history, shared contract with the
 * GPU path, restated here independently):
 *   key     = (seed low 32 bits, seed high 32 bits)
 *   counter = (block n, history id low, history id high, instance id)
 *   block n yields 4 words consumed in order, then n advances.
 *   u = (2*(x >> 9) + 1) * 2^-24  -- 24 significant bits, so the value is the
 *   same in binary32 and binary64 and lies strictly inside (0, 1).
 */
#include "oracle.h"

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

double orc_u01(uint32_t x)
{
    return (double)(2u * (x >> 9) + 1u) * (1.0 / 16777216.0);
}

void orc_stream_words(uint64_t seed, uint64_t hid, uint32_t inst, int n_words, uint32_t *out)
{
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t ctr[4] = { 0u, (uint32_t)hid, (uint32_t)(hid >> 32), inst };
    uint32_t block[4];
    for (int i = 0; i < n_words; ++i) {
        if (i % 4 == 0) {
            ctr[0] = (uint32_t)(i / 4);
            orc_philox4x32_10(ctr, key, block);
        }
        out[i] = block[i % 4];
    }
}
