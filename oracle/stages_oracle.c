/*
 * CPU ORACLE for the stages that follow the block sort -- TEST INFRASTRUCTURE.
 *
 * Only the tests, the smoke check and the benchmark's CPU arms may load this
 * library (it is built into the same liboracle.so as the block-sort oracle).
 * It shares no code with the CUDA path.
 *
 * Each routine is the plain sequential definition of its stage; the GPU
 * methods the paper describes reach exactly these results:
 *   run-length encoding (Section 3.2, Fig. 1 and Fig. 2): a block becomes its
 *     maximal runs, each a (byte, length) pair, in order; decoding repeats
 *     every byte `length` times. Runs never cross a block boundary.
 *   move-to-front encoding (Section 3.3): a list of the 256 byte values starts
 *     in ascending order; every input byte is replaced by its current position
 *     in the list and then moved to the front. Decoding replays the list.
 *   variable-length encoding (Section 3.4, Fig. 3): every byte is replaced by
 *     its codeword from a given table (code value, length in bits); codewords
 *     are written one after another, most significant bit first, into a bit
 *     stream whose bit p is bit 7 - (p mod 8) of byte p / 8. A codeword's
 *     first bit position is the sum of the lengths before it (the exclusive
 *     prefix sum of Fig. 3).
 *
 * Parity pins (tests/test_oracle_stages.py): the worked examples of Fig. 1,
 * Fig. 2 and Fig. 3 (tests/golden/), decode(encode(x)) == x, brute-force
 * properties (maximal runs, list contents, bit counts) and closed forms.
 */
#include <stdint.h>
#include <string.h>

/* Runs of S[0..n): chars[k], lens[k] for k < returned count. */
int64_t oracle_rle_encode(const uint8_t *S, int64_t n, uint8_t *chars, uint32_t *lens) {
    int64_t k = 0;
    int64_t i = 0;
    while (i < n) {
        int64_t j = i + 1;
        while (j < n && S[j] == S[i]) ++j;
        chars[k] = S[i];
        lens[k] = (uint32_t)(j - i);
        ++k;
        i = j;
    }
    return k;
}

/* Expands `runs` (byte, length) pairs into out; returns the bytes written. */
int64_t oracle_rle_decode(const uint8_t *chars, const uint32_t *lens, int64_t runs, uint8_t *out) {
    int64_t o = 0;
    for (int64_t k = 0; k < runs; ++k)
        for (uint32_t r = 0; r < lens[k]; ++r) out[o++] = chars[k];
    return o;
}

void oracle_mtf_encode(const uint8_t *S, int64_t n, uint8_t *out) {
    uint8_t list[256];
    for (int c = 0; c < 256; ++c) list[c] = (uint8_t)c;
    for (int64_t i = 0; i < n; ++i) {
        int p = 0;
        while (list[p] != S[i]) ++p;
        out[i] = (uint8_t)p;
        memmove(list + 1, list, (size_t)p);
        list[0] = S[i];
    }
}

void oracle_mtf_decode(const uint8_t *in, int64_t n, uint8_t *out) {
    uint8_t list[256];
    for (int c = 0; c < 256; ++c) list[c] = (uint8_t)c;
    for (int64_t i = 0; i < n; ++i) {
        const int p = in[i];
        const uint8_t c = list[p];
        out[i] = c;
        memmove(list + 1, list, (size_t)p);
        list[0] = c;
    }
}

/* Bit stream of S[0..n) under the table (code[c] right-aligned, len[c] in
 * 1..32 bits). out must hold ceil(total bits / 8) zeroed bytes; returns the
 * number of bits. pos, if not NULL, receives each codeword's first bit. */
int64_t oracle_vle_encode(const uint8_t *S, int64_t n, const uint32_t *code, const uint8_t *len, uint8_t *out,
                          uint64_t *pos) {
    uint64_t p = 0;
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t c = code[S[i]];
        const int l = len[S[i]];
        if (pos) pos[i] = p;
        for (int b = l - 1; b >= 0; --b, ++p)
            if ((c >> b) & 1u) out[p >> 3] |= (uint8_t)(0x80u >> (p & 7));
    }
    return (int64_t)p;
}
