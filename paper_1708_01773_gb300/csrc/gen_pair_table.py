"""Writes the node-pair table of the tensor-core epilogue (fe_pair_table.h).

The epilogue of k_cell_tc gives each thread one node pair (a, b), a <= b < 27,
which loads G[(i,a),(j,b)] (row stride 100 floats) and stores K^e entries
(i,a),(j,b) and (j,b),(i,a) (row stride 84 floats) for i, j = 0..2. The 32
threads of a warp hit 32 distinct shared-memory banks in all three accesses
when, within the warp's group of pairs, the residues mod 32 of 4a + b (load),
20a + b (direct store) and 20b + a (transposed store) are all distinct. This
script partitions the 378 pairs into 15 such groups (randomised greedy
packing, fixed seeds, deterministic) and writes them as a C table, one row of
32 entries per group, 0xffff marking an empty lane.
"""
import os
import random

NB, WARP, GROUPS = 27, 32, 15


def keys(a, b):
    return ((4 * a + b) % 32, (20 * a + b) % 32, (20 * b + a) % 32)


def search():
    pairs = [(a, b) for a in range(NB) for b in range(a, NB)]
    for seed in range(100000):
        rng = random.Random(seed)
        order = pairs[:]
        rng.shuffle(order)
        groups = [[] for _ in range(GROUPS)]
        used = [[set(), set(), set()] for _ in range(GROUPS)]
        for a, b in order:
            k = keys(a, b)
            cands = [g for g in range(GROUPS)
                     if len(groups[g]) < WARP and all(k[t] not in used[g][t] for t in range(3))]
            if not cands:
                break
            g = max(cands, key=lambda g: (len(groups[g]), rng.random()))
            groups[g].append((a, b))
            for t in range(3):
                used[g][t].add(k[t])
        else:
            return seed, groups
    raise RuntimeError("no partition found")


def main():
    seed, groups = search()
    rows = []
    for g in groups:
        ent = [f"0x{(a << 8) | b:04x}" for a, b in g] + ["0xffff"] * (WARP - len(g))
        rows.append("    {" + ", ".join(ent) + "},")
    text = ("// Generated by gen_pair_table.py (seed %d): node pairs a <= b of the Q2\n"
            "// tensor-core epilogue, one row of 32 lanes per warp-round group, entry\n"
            "// (a << 8) | b, 0xffff = idle lane. Within a row the residues mod 32 of\n"
            "// 4a + b, 20a + b and 20b + a are distinct (conflict-free shared memory).\n"
            "#pragma once\n#include <cstdint>\n\nnamespace feasm {\nnamespace tc {\n\n"
            "constexpr int PAIR_GROUPS = %d;\n"
            "__device__ const uint16_t kPairTable[PAIR_GROUPS][32] = {\n%s\n};\n\n"
            "}  // namespace tc\n}  // namespace feasm\n") % (seed, GROUPS, "\n".join(rows))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fe_pair_table.h")
    with open(out, "w") as f:
        f.write(text)
    print("wrote", out, "seed", seed)


if __name__ == "__main__":
    main()
