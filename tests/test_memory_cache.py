"""The device memory cache's reuse policy (Sec. III-C memory cache: reuse a
free buffer whose capacity covers the request), exercised on host tensors."""
import pytest

torch = pytest.importorskip("torch")

from paper_2109_14704_gb300.serving import DeviceMemoryCache  # noqa: E402


def test_reuse_smallest_sufficient_buffer():
    c = DeviceMemoryCache(torch.device("cpu"))
    a = c.allocate(100)
    b = c.allocate(400)
    assert c.misses == 2 and c.in_use == 500 * 8 and c.reserved == 500 * 8
    c.free(*a)
    c.free(*b)
    assert c.in_use == 0
    cap, t = c.allocate(90)            # fits both; the smaller one is taken
    assert cap == 100 and c.hits == 1
    cap2, t2 = c.allocate(300)         # only the larger one fits
    assert cap2 == 400 and c.hits == 2
    cap3, _ = c.allocate(500)          # nothing fits: a new buffer
    assert cap3 == 500 and c.misses == 3 and c.reserved == 1000 * 8
    assert c.in_use == 1000 * 8


def test_allocate_within_budget_evicts_free_buffers():
    c = DeviceMemoryCache(torch.device("cpu"))
    a = c.allocate(100)
    b = c.allocate(200)
    c.free(*a)
    c.free(*b)
    assert c.reserved == 300 * 8
    # 150 words reuse the 200-word buffer: no growth, fits a 300-word budget
    got = c.allocate_within([150], limit_bytes=300 * 8)
    assert got is not None and got[0][0] == 200 and c.reserved == 300 * 8
    c.free(*got[0])
    # 250 words need new memory; evicting free buffers makes room
    got = c.allocate_within([250], limit_bytes=300 * 8)
    assert got is not None and c.reserved <= 300 * 8 and c.evicted >= 1
    # nothing free to evict and no room: refused, nothing allocated
    before = (c.reserved, c.in_use)
    assert c.allocate_within([100], limit_bytes=300 * 8) is None
    assert (c.reserved, c.in_use) == before


def test_size_classes_round_up_and_serve_neighbours():
    c = DeviceMemoryCache(torch.device("cpu"), size_classes=True)
    for words in (1000, 4096, 5000, 123457, 1 << 20):
        cap = c._capacity(words)
        # the next quarter-octave size (rounded to 256 words): at most 19 % slack
        assert words <= cap <= words * 2 ** 0.25 + 256 and cap % 256 == 0
    assert c._capacity(100) == 100            # small requests stay exact
    a = c.allocate(5000)
    c.free(*a)
    b = c.allocate(5100)                      # a neighbouring size reuses it
    assert b[0] == a[0] and c.hits == 1 and c.misses == 1


def test_many_free_buffers_pick_smallest_sufficient():
    c = DeviceMemoryCache(torch.device("cpu"))
    bufs = [c.allocate(w) for w in range(1000, 3000, 7)]
    for b in reversed(bufs):
        c.free(*b)
    cap, _ = c.allocate(2000)
    assert cap == min(w for w in range(1000, 3000, 7) if w >= 2000)
    assert [x for x, _ in c.free_list] == sorted(x for x, _ in c.free_list)
