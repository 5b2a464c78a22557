"""The bench's algorithmic work counts, on which every roofline fraction
rests, against counts worked out by hand from the definitions (host only).

Tree hash of a P976 ciphertext (16 n + 128 = 15744 bytes): 15 chunks of
1024 bytes at 1024 // 136 + 1 = 8 permutations each, a last chunk of 384
bytes at 3, and the root over 16 digests (512 bytes) at 4: 127.  A P640
ciphertext (10368 bytes): 10 x 8 + 1 (128 bytes) + 3 (11 digests, 352
bytes) = 84."""
import types

import bench


def test_keccak_permutations_of_the_tree_hash():
    assert bench.keccak_perms(16 * 976 + 128) == 127
    assert bench.keccak_perms(16 * 640 + 128) == 84
    # a message of whole chunks has no short leaf: 2 x 8 + root (64 B) 1
    assert bench.keccak_perms(2048) == 17
    # one block's boundary: 135 bytes take one permutation, 136 two
    assert bench.keccak_perms(135) == 1 + 1
    assert bench.keccak_perms(136) == 2 + 1


def test_step_work_of_the_batched_p976_workload():
    p = types.SimpleNamespace(n=976)
    w = bench.algorithmic(p, 4096)
    # GEMM: 2 launches x 2 limbs x 2 flops x 32768 rows x 984 columns x 976
    assert w["k_gemm_tc"][1] == 2 * (2 * 2 * 32768 * 984 * 976)
    # noise: Encaps and Decaps x 2 bytes x (S' 8n + E' 8n + E'' 64 samples)
    assert w["k_noise"][1] == 2 * 2 * (16 * 976 + 64) * 4096
    # tree: H(c) in Encaps and Decaps, and Encaps' K (one permutation each)
    assert w["k_tree"][1] == 2 * 4096 * 127 + 4096 == 1044480
