"""Pin of the seeded input generator shared by the oracle and the CUDA path
(cdg2_inputs.SplitMix64): the first outputs for seed 1234567 are the
generator's published test vector (the reference implementation of
SplitMix64, Steele, Lea and Flood, OOPSLA 2014, as distributed with
xorshift/xoshiro by Vigna), and uniform() takes the top 53 bits."""
import cdg2_inputs as I

PUBLISHED_SEED_1234567 = (6457827717110365317, 3203168211198807973, 9817491932198370423,
                          4593380528125082431, 16408922859458223821)


def test_splitmix64_matches_its_published_outputs():
    g = I.SplitMix64(1234567)
    assert tuple(g.next_u64() for _ in range(5)) == PUBLISHED_SEED_1234567


def test_uniform_is_the_top_53_bits():
    g, h = I.SplitMix64(1234567), I.SplitMix64(1234567)
    for v in PUBLISHED_SEED_1234567:
        u = g.uniform()
        assert u == (v >> 11) / 2.0 ** 53 and 0.0 <= u < 1.0
        assert h.next_u64() == v
