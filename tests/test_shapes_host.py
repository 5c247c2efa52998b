"""The transform shapes the library lists and accepts, on the CPU (no device
work: he_ntt_shapes and he_ntt_set_shape are host calls). For every degree
2^10 .. 2^16: the default comes first, every listed shape is a valid split
of the transform (blocks of at most N words, clusters of 1 to 16 CTAs,
radix-8 or radix-16 register rounds, at most 1024 threads per CTA), every
listed shape is accepted for either direction and both launch forms, a shape
that is not listed is refused with HE_EUNSUPPORTED, and the all-zero call
restores the default. The shapes themselves are checked against the oracle
on the GPU by tests/test_gpu_ntt.py."""
import pytest

from paper_2109_14704_gb300 import he

DEGREES = range(10, 17)


@pytest.fixture(autouse=True)
def _restore_defaults():
    yield
    for log_n in DEGREES:
        he.ntt_set_shape(1 << log_n, 0, 0, 0)


@pytest.mark.parametrize("log_n", DEGREES)
def test_listed_shapes_are_valid_splits(log_n):
    N = 1 << log_n
    shapes = he.ntt_shapes(N)
    assert shapes and len(set(shapes)) == len(shapes)
    for lb, le, occ in shapes:
        assert 10 <= lb <= log_n, (lb, le)
        assert 1 <= N >> lb <= 16, (lb, le)                  # cluster of at most 16 CTAs
        assert le in (3, 4), (lb, le)                        # radix-8 or radix-16 rounds
        assert (1 << (lb - le)) <= 1024, (lb, le)            # threads per CTA
        assert 0 <= occ <= 16, occ                           # CTAs per SM the build is compiled for
    assert shapes[0][2] == 0                                 # the default: the shape's own register budget


@pytest.mark.parametrize("log_n", DEGREES)
def test_every_listed_shape_is_accepted_and_others_refused(log_n):
    N = 1 << log_n
    shapes = he.ntt_shapes(N)
    for lb, le, occ in shapes:
        for direction in (he.FORWARD, he.INVERSE, he.BOTH):
            for pers in (0, 1):
                he.ntt_set_shape(N, lb, le, pers, direction=direction, ctas_per_sm=occ)
    listed = set(shapes)
    for lb in range(9, log_n + 2):
        for le in (2, 3, 4, 5):
            for occ in (0, 1, 3, 7):
                if (lb, le, occ) in listed or (lb, le, occ) == (0, 0, 0):
                    continue
                with pytest.raises(he.HeError) as e:
                    he.ntt_set_shape(N, lb, le, 0, ctas_per_sm=occ)
                assert e.value.status in (he.HE_EUNSUPPORTED, he.HE_EINVAL), (lb, le, occ)
    he.ntt_set_shape(N, 0, 0, 0)                             # the default again


def test_degrees_outside_the_built_range_are_refused():
    for N in (1 << 9, 1 << 17, 3000):
        with pytest.raises(he.HeError):
            he.ntt_shapes(N)
        with pytest.raises(he.HeError):
            he.ntt_set_shape(N, 0, 0, 0)
