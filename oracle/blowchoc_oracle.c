/*
 * Oracle for Blocked Bloom filters with choices (BlowChoc filters).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, single-threaded
 * CPU statement of what the GPU path computes. Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it. It
 * shares no code, header, table or constant generator with the CUDA
 * library, and it never calls into it.
 *
 * Everything is written bit by bit, the way the paper states it: a block is
 * 512 single bits, a key's bit set F(x) is a boolean array over [512], loads
 * are counted one bit at a time, and costs are evaluated in IEEE double
 * with the paper's formulas. No popcount, no word-level masks.
 *
 * Paper: J. E. Schmitz, J. Zentgraf, S. Rahmann, "Blocked Bloom Filters with
 * Choices", arXiv 2501.18977.
 *
 * Readings where the paper is silent (each listed in the design notes):
 *  - hash multipliers come from a splitmix64 stream seeded with the filter's
 *    seed, forced odd, redrawn until coprime to the hash range; order: the c
 *    block multipliers, then the k bit multipliers;
 *  - keys are u = 64-bit, so the xor-fold shift is 32;
 *  - bit p of block b is bit (p mod 64) of 64-bit word 8b + p/64;
 *  - ties between choices go to the lowest choice index;
 *  - a batch of B keys chooses against the bits present at the batch start
 *    and is OR-ed in afterwards (B = 1 is the paper's one-key-at-a-time
 *    insertion).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_BLOCK_BITS 512u

enum { ORC_COST_MIX = 0, ORC_COST_LA = 1, ORC_COST_EXP = 2, ORC_COST_TABLE = 3 };

/* A cost given as a table over (load L, new bits a): cost = table[L (k+1) + a]
 * with L = j - a. Used for costs that are not among Eq. 4-6 (a learned cost). */
static const double *orc_table = NULL;
static uint32_t orc_table_k = 0;

void orc_set_cost_table(const double *table, uint32_t k)
{
    orc_table = table;
    orc_table_k = k;
}

/* Bit selection (Section 3.3): 0 = random, 1 = distinct (Appendix B). */
static int orc_bitsel = 0;

void orc_set_bitsel(int mode) { orc_bitsel = mode; }

/* splitmix64 (Steele, Lea and Flood, OOPSLA 2014): add the golden-ratio
 * increment to the state, then apply the variant-13 finaliser of MurmurHash3
 * as published with the generator. Used here only to draw hash multipliers. */
uint64_t orc_splitmix64_next(uint64_t *state)
{
    uint64_t z = (*state += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static uint64_t orc_gcd(uint64_t a, uint64_t b)
{
    while (b != 0) {
        uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

static int orc_is_pow2(uint64_t b) { return b != 0 && (b & (b - 1)) == 0; }

static unsigned orc_log2(uint64_t b)
{
    unsigned r = 0;
    while (b > 1) {
        b >>= 1;
        r++;
    }
    return r;
}

/* Linear hash of Section 3.4 ("Hash functions") with u = 64:
 *   y = (a x) mod 2^64;
 *   b a power of two:       the log2(b) most significant bits of y;
 *   b even, not a power:    (y xor (y >> 32)) mod b;
 *   b odd:                  y mod b.
 * A range of b = 1 has log2 b = 0 significant bits, so the value is 0. */
uint64_t orc_hash(uint64_t a, uint64_t x, uint64_t b)
{
    uint64_t y = a * x; /* unsigned arithmetic wraps mod 2^64 */
    if (orc_is_pow2(b)) {
        unsigned lg = orc_log2(b);
        if (lg == 0)
            return 0;
        return (y >> (64u - lg)) % b;
    }
    if ((b & 1u) == 0)
        y = y ^ (y >> 32);
    return y % b;
}

/* Section 3.4: "a is a random large integer, and a and b are coprime".
 * Draw a_1..a_c for the block hashes (range M) and then a'_1..a'_k for the
 * bit hashes (range 512) from one splitmix64 stream. Returns 0, or -1 on
 * bad arguments. */
int orc_derive_multipliers(uint64_t seed, uint64_t M, uint32_t k, uint32_t c,
                           uint64_t *a_block, uint64_t *a_bit)
{
    if (M == 0 || k == 0 || k > 32 || c == 0 || c > 3)
        return -1;
    uint64_t state = seed;
    for (uint32_t i = 0; i < c; i++) {
        uint64_t a;
        do {
            a = orc_splitmix64_next(&state) | 1u;
        } while (orc_gcd(a, M) != 1);
        a_block[i] = a;
    }
    for (uint32_t i = 0; i < k; i++) {
        /* random bits hash into [512]; distinct bits: f_{i+1} into [512 - i] */
        uint64_t range = orc_bitsel ? ORC_BLOCK_BITS - i : ORC_BLOCK_BITS;
        uint64_t a;
        do {
            a = orc_splitmix64_next(&state) | 1u;
        } while (orc_gcd(a, range) != 1);
        a_bit[i] = a;
    }
    return 0;
}

/* Insertion cost of a block for a key, with j = total set bits after the
 * insertion and a = newly set bits (Section 3.2; Appendix A):
 *   MIX (Eq. 5):  sigma k (j/256)^k + a
 *   LA  (Eq. 6):  k ((j + mu k)/256)^k + a
 *   EXP (Eq. 4):  beta^(j/128) + a/k
 * param is sigma, mu or beta. Evaluated in double in exactly this order. */
double orc_cost(int kind, double param, uint32_t k, uint32_t j, uint32_t a)
{
    double dk = (double)k;
    if (kind == ORC_COST_TABLE)
        return (orc_table != NULL && k == orc_table_k) ? orc_table[(j - a) * (k + 1) + a] : NAN;
    if (kind == ORC_COST_MIX)
        return (param * dk) * pow((double)j / 256.0, dk) + (double)a;
    if (kind == ORC_COST_LA)
        return dk * pow(((double)j + param * dk) / 256.0, dk) + (double)a;
    return pow(param, (double)j / 128.0) + (double)a / dk;
}

static int orc_get_bit(const uint64_t *words, uint64_t b, uint32_t p)
{
    return (int)((words[8u * b + p / 64u] >> (p % 64u)) & 1u);
}

static void orc_set_bit(uint64_t *words, uint64_t b, uint32_t p)
{
    words[8u * b + p / 64u] |= (uint64_t)1 << (p % 64u);
}

/* F(x) = { f_i(x) : i = 1..k } (Eq. 3), random bit selection (Section 3.3):
 * each f_i is the linear hash into [512]. Collisions make |F| < k. */
static void orc_bitset(const uint64_t *a_bit, uint32_t k, uint64_t x,
                       unsigned char inF[ORC_BLOCK_BITS])
{
    memset(inF, 0, ORC_BLOCK_BITS);
    if (!orc_bitsel) {
        for (uint32_t i = 0; i < k; i++)
            inF[orc_hash(a_bit[i], x, ORC_BLOCK_BITS)] = 1;
        return;
    }
    /* Distinct bit selection (Appendix B, Fig. 9): f_i hashes into
     * [512 - i + 1]; it is then incremented as long as some earlier address,
     * scanned in ascending order, is smaller than or equal to its current
     * value, and inserted into the sorted list of addresses (insertion sort).
     * The result is a uniform k-subset of [512]. */
    uint32_t sorted[32];
    uint32_t nsorted = 0;
    for (uint32_t i = 0; i < k; i++) {
        uint32_t f = (uint32_t)orc_hash(a_bit[i], x, ORC_BLOCK_BITS - i);
        uint32_t pos = 0;
        while (pos < nsorted && sorted[pos] <= f) {
            f++;
            pos++;
        }
        for (uint32_t t = nsorted; t > pos; t--)
            sorted[t] = sorted[t - 1];
        sorted[pos] = f;
        nsorted++;
    }
    for (uint32_t t = 0; t < nsorted; t++)
        inF[sorted[t]] = 1;
}

/* Exported for tests: the distinct-selection shift rule applied to given raw
 * values raw[i] in [512 - i] (Appendix B); out receives the final addresses
 * in the order the raw values are given. */
void orc_distinct_from_raw(const uint32_t *raw, uint32_t k, uint32_t *out)
{
    uint32_t sorted[32];
    uint32_t nsorted = 0;
    for (uint32_t i = 0; i < k; i++) {
        uint32_t f = raw[i];
        uint32_t pos = 0;
        while (pos < nsorted && sorted[pos] <= f) {
            f++;
            pos++;
        }
        for (uint32_t t = nsorted; t > pos; t--)
            sorted[t] = sorted[t - 1];
        sorted[pos] = f;
        nsorted++;
        out[i] = f;
    }
}

/* Exported for tests: the positions of F(x), ascending; returns |F(x)|. */
uint32_t orc_bit_positions(const uint64_t *a_bit, uint32_t k, uint64_t x,
                           uint32_t *out)
{
    unsigned char inF[ORC_BLOCK_BITS];
    uint32_t n = 0;
    orc_bitset(a_bit, k, x, inF);
    for (uint32_t p = 0; p < ORC_BLOCK_BITS; p++)
        if (inF[p])
            out[n++] = p;
    return n;
}

/* |F'|: the number of set bits of block b, counted one bit at a time. */
static uint32_t orc_block_load(const uint64_t *words, uint64_t b)
{
    uint32_t L = 0;
    for (uint32_t p = 0; p < ORC_BLOCK_BITS; p++)
        L += (uint32_t)orc_get_bit(words, b, p);
    return L;
}

/* a = |F(x) \ F'|: the bits of F(x) that block b does not hold yet. */
static uint32_t orc_new_bits(const uint64_t *words, uint64_t b,
                             const unsigned char inF[ORC_BLOCK_BITS])
{
    uint32_t a = 0;
    for (uint32_t p = 0; p < ORC_BLOCK_BITS; p++)
        if (inF[p] && !orc_get_bit(words, b, p))
            a++;
    return a;
}

/* Choice for one key against the current bits (Section 3.2).
 * Returns -1 if some candidate block already holds all of F(x) (nothing to
 * change), otherwise the index i in [0, c) of the block h_{i+1}(x) of least
 * cost, scanning i upwards with a strict comparison so that ties go to the
 * lowest index. With c = 1 there is no cost evaluation: the only block. */
static int orc_choose(const uint64_t *words, uint64_t M, uint32_t k, uint32_t c,
                      int kind, double param, const uint64_t *a_block,
                      const unsigned char inF[ORC_BLOCK_BITS], uint64_t x)
{
    uint64_t blk[3];
    uint32_t a[3];
    for (uint32_t i = 0; i < c; i++) {
        blk[i] = orc_hash(a_block[i], x, M);
        a[i] = orc_new_bits(words, blk[i], inF);
        if (a[i] == 0)
            return -1;
    }
    if (c == 1)
        return 0;
    int best = -1;
    double best_cost = 0.0;
    for (uint32_t i = 0; i < c; i++) {
        uint32_t L = orc_block_load(words, blk[i]);
        double cost = orc_cost(kind, param, k, L + a[i], a[i]);
        if (best < 0 || cost < best_cost) {
            best = (int)i;
            best_cost = cost;
        }
    }
    return best;
}

/* Batch-synchronous insertion of keys[0..n) in batches of B keys.
 * For each batch, every key first takes its choice against the filter as it
 * stands at the batch start; only then are the chosen bit sets OR-ed in.
 * B = 1 is exactly the paper's sequential insertion (Section 3.1/3.2).
 * choice_out (optional, n entries): -1 = skipped, else the chosen index.
 * Returns 0, or -1 on bad arguments / allocation failure. */
int orc_insert(uint64_t *words, uint64_t M, uint32_t k, uint32_t c, int kind,
               double param, const uint64_t *a_block, const uint64_t *a_bit,
               const uint64_t *keys, uint64_t n, uint64_t B,
               int8_t *choice_out, uint64_t *inserted, uint64_t *skipped)
{
    if (M == 0 || k == 0 || k > 32 || c == 0 || c > 3 || B == 0)
        return -1;
    uint64_t cap = B < n ? B : n;
    int8_t *choice = choice_out;
    int8_t *tmp = NULL;
    if (choice == NULL && n > 0) {
        tmp = (int8_t *)malloc(cap);
        if (tmp == NULL)
            return -1;
    }
    unsigned char inF[ORC_BLOCK_BITS];
    uint64_t n_ins = 0, n_skip = 0;
    for (uint64_t s = 0; s < n; s += B) {
        uint64_t e = (n - s) < B ? n : s + B;
        int8_t *ch = choice ? choice + s : tmp;
        /* choose against the snapshot at the batch start */
        for (uint64_t t = s; t < e; t++) {
            orc_bitset(a_bit, k, keys[t], inF);
            ch[t - s] = (int8_t)orc_choose(words, M, k, c, kind, param, a_block,
                                           inF, keys[t]);
        }
        /* then set the bits in the chosen blocks */
        for (uint64_t t = s; t < e; t++) {
            if (ch[t - s] < 0) {
                n_skip++;
                continue;
            }
            n_ins++;
            uint64_t b = orc_hash(a_block[(int)ch[t - s]], keys[t], M);
            orc_bitset(a_bit, k, keys[t], inF);
            for (uint32_t p = 0; p < ORC_BLOCK_BITS; p++)
                if (inF[p])
                    orc_set_bit(words, b, p);
        }
    }
    free(tmp);
    if (inserted)
        *inserted = n_ins;
    if (skipped)
        *skipped = n_skip;
    return 0;
}

/* Membership query (Section 3.1): true iff all bits of F(x) are set in at
 * least one of the c candidate blocks. Result bit t of the bitmap is key t,
 * least significant bit first within 64-bit words; bits past n are zero.
 * first_out (optional, n entries): the 1-based index of the first candidate
 * block that holds F(x), or 0 if none. */
int orc_query(const uint64_t *words, uint64_t M, uint32_t k, uint32_t c,
              const uint64_t *a_block, const uint64_t *a_bit,
              const uint64_t *keys, uint64_t n, uint64_t *bitmap,
              uint8_t *first_out)
{
    if (M == 0 || k == 0 || k > 32 || c == 0 || c > 3)
        return -1;
    memset(bitmap, 0, ((n + 63) / 64) * sizeof(uint64_t));
    unsigned char inF[ORC_BLOCK_BITS];
    for (uint64_t t = 0; t < n; t++) {
        orc_bitset(a_bit, k, keys[t], inF);
        int hit = 0;
        for (uint32_t i = 0; i < c && !hit; i++) {
            uint64_t b = orc_hash(a_block[i], keys[t], M);
            int all = 1;
            for (uint32_t p = 0; p < ORC_BLOCK_BITS && all; p++)
                if (inF[p] && !orc_get_bit(words, b, p))
                    all = 0;
            if (all)
                hit = (int)i + 1;
        }
        if (hit)
            bitmap[t / 64] |= (uint64_t)1 << (t % 64);
        if (first_out)
            first_out[t] = (uint8_t)hit;
    }
    return 0;
}

/* Load histogram (Appendix C, Fig. 8): hist[L] = number of blocks holding
 * exactly L set bits, L = 0..512. Also returns the total number of set bits. */
uint64_t orc_histogram(const uint64_t *words, uint64_t M, uint64_t *hist)
{
    uint64_t total = 0;
    memset(hist, 0, (ORC_BLOCK_BITS + 1) * sizeof(uint64_t));
    for (uint64_t b = 0; b < M; b++) {
        uint32_t L = orc_block_load(words, b);
        hist[L]++;
        total += L;
    }
    return total;
}

/* Exported for tests: load |F'| of block b and new bits a of key x there. */
void orc_block_terms(const uint64_t *words, uint64_t b, const uint64_t *a_bit,
                     uint32_t k, uint64_t x, uint32_t *L, uint32_t *a)
{
    unsigned char inF[ORC_BLOCK_BITS];
    orc_bitset(a_bit, k, x, inF);
    *L = orc_block_load(words, b);
    *a = orc_new_bits(words, b, inF);
}
