"""Host tests of the render server's admission by HBM footprint (no GPU).

The scenes, frames and device are stand-ins whose workspace sizes and phase durations
the test sets, so the interleavings that matter are reproduced on the CPU: a request
whose tile lists become known only after its count phase, while another request was
admitted into the budget it had left free.
"""
import time

from paper_1606_04427_gb300 import serve


class _Device:
    def bind(self):
        pass

    def free_bytes(self):
        return 1 << 30

    def stream(self):
        return object()

    def image(self, height, width, stream):
        return None

    def synchronize(self, stream):
        pass


class _Frame:
    def __init__(self, fixed, var, render_s):
        self.fixed_bytes, self.var_bytes, self.pairs = fixed, var, 1
        self.render_s = render_s

    def render(self, out=None, stream=None):
        time.sleep(self.render_s)

    def close(self):
        pass


class _Scene:
    n = 1000

    def __init__(self, fixed, var, count_s, render_s):
        self.fixed, self.var, self.count_s, self.render_s = fixed, var, count_s, render_s

    def frame_fixed_bytes(self, cam, params=None):
        return self.fixed

    def prepare(self, cam, params=None, stream=None):
        time.sleep(self.count_s)
        return _Frame(self.fixed, self.var, self.render_s)


class _Camera:
    width = 1
    height = 1  # 12 image bytes


def _run(scenes, order, budget, slots=2, gap_s=0.0):
    srv = serve.Server(scenes, slots=slots, hbm_budget=budget, device=_Device())
    try:
        for i in order:
            srv.submit(i, _Camera())
            time.sleep(gap_s)
        srv.wait_all(timeout=30)
    finally:
        srv.close()
    assert not srv.errors, srv.errors
    assert len(srv.done) == len(order)
    return srv


def test_lists_that_no_longer_fit_send_the_request_back():
    """A (lists 800 B, slow count phase) is admitted alone with 112 B; B (212 B in all) is
    admitted into the budget A left free and renders for a while.  When A's lists become
    known they no longer fit beside B: A gives its bytes back and waits, and is admitted
    again with its full footprint once B is done.  The reservations never pass the budget."""
    a = _Scene(fixed=100, var=800, count_s=0.2, render_s=0.01)
    b = _Scene(fixed=100, var=100, count_s=0.0, render_s=0.5)
    srv = _run([a, b], [0, 1], budget=1000, gap_s=0.02)
    assert srv.peak_reserved <= 1000, srv.peak_reserved
    assert srv.requeued >= 1
    got = {c.set_index: c for c in srv.done}
    assert got[0].reserved_bytes == 912 and got[1].reserved_bytes == 212
    assert got[0].allocated_bytes == got[0].reserved_bytes


def test_a_request_larger_than_the_budget_runs_alone():
    """A footprint above the whole budget is still served, with nothing else in flight."""
    big = _Scene(fixed=100, var=2000, count_s=0.0, render_s=0.01)
    small = _Scene(fixed=100, var=100, count_s=0.0, render_s=0.01)
    srv = _run([big, small], [0, 1, 1], budget=1000, slots=3)
    got = [c for c in srv.done if c.set_index == 0]
    assert got[0].reserved_bytes == 2112
    assert srv.peak_reserved == 2112  # the large request ran with nothing beside it


def test_reservations_stay_within_the_budget_under_a_mixed_stream():
    """Forty requests of four sizes over four slots: every one completes, each reserved
    exactly what its frame and image take, and the sum never passed the budget."""
    scenes = [_Scene(fixed=50 + 10 * k, var=100 * (k + 1), count_s=0.002 * k, render_s=0.003) for k in range(4)]
    order = [(7 * i) % 4 for i in range(40)]
    srv = _run(scenes, order, budget=900, slots=4)
    assert srv.peak_reserved <= 900
    for c in srv.done:
        assert c.reserved_bytes == c.allocated_bytes
