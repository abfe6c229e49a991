"""Pins of the oracle's per-frame stage order (``oracle.frontend.step``,
Sec. III-B) on a hand-worked two-frame case.

The tracker, detector and pyramid are replaced by stand-ins whose results are
fixed by hand, so that what is checked is the step's own logic: which
pyramids each stage reads, that tracking comes before detection and feeds it
the per-cell counts of the surviving camera-0 tracks, the order of the new
lists (survivors, then new keypoints), the numbering of new ids, that camera 1
receives only the successful matches at their matched positions, and the
truncation to the capacity. Every expected value below is worked out in the
comments from the stand-ins' rules."""
import numpy as np
import pytest

from oracle import frontend as ofe

W, H, CW, CH = 100, 60, 50, 30          # 2 x 2 cells
CANDIDATE = {0: (10.0, 10.0), 1: (60.0, 10.0), 2: (10.0, 40.0), 3: (60.0, 40.0)}


def _frame(tag):
    """Two 60x100 images whose pixel (0, 0) identifies the frame and camera."""
    f = np.zeros((2, H, W), np.uint8)
    f[0, 0, 0] = 10 * tag
    f[1, 0, 0] = 10 * tag + 1
    return f


class Stand:
    """Stand-ins for pyramid, track and detect_grid with hand-set rules."""

    def __init__(self):
        self.calls = []

    def pyramid(self, img, n_levels, round_mode):
        return ("pyr", int(img[0, 0]))

    def track(self, src, dst, xy, init=None, **kw):
        xy = np.asarray(xy, np.float64)
        n = len(xy)
        s, d = src[1], dst[1]
        self.calls.append(("track", s, d, n))
        status = np.zeros(n, np.uint8)
        warp = np.zeros((n, 3))
        if s % 10 == 0 and d == s + 1:                 # stereo: cam0 -> cam1, same frame
            warp[:, :2] = xy - [7.0, 0.0]              # disparity 7 px
            status[(xy[:, 0] == 60) & (xy[:, 1] == 40)] = 5      # FB_FAIL
        elif s % 10 == 0:                              # temporal camera 0
            warp[:, :2] = xy + [1.0, 1.0]
            status[(xy[:, 0] == 10) & (xy[:, 1] == 40)] = 2      # OOB_WARP
        else:                                          # temporal camera 1
            warp[:, :2] = xy + [2.0, 0.0]
            status[(xy[:, 0] == 3) & (xy[:, 1] == 40)] = 2
        return {"status": status, "warp": warp, "fb_dist": np.zeros(n), "margin": np.ones(n)}

    def detect_grid(self, img, cw, ch, k=1, thresholds=None, border=9, occupancy=None):
        self.calls.append(("detect", int(img[0, 0]), occupancy.tolist()))
        pts = [CANDIDATE[c] for c in range(4) if occupancy[c] < k]
        return (np.array(pts, np.float32).reshape(-1, 2),
                np.full(len(pts), 50, np.int16))


@pytest.fixture
def stand(monkeypatch):
    st = Stand()
    monkeypatch.setattr(ofe, "pyramid", st.pyramid)
    monkeypatch.setattr(ofe, "track", st.track)
    monkeypatch.setattr(ofe, "detect_grid", st.detect_grid)
    return st


P = ofe.Params(n_levels=2, cell_w=CW, cell_h=CH, k=1)


def test_two_frames_by_hand(stand):
    s = ofe.StreamState()
    # frame 1: no previous pyramid -> no tracking; every cell free; the four
    # candidates are new (ids 0..3); matching moves them by -7 px and fails
    # (60, 40), so camera 1 holds ids 0, 1, 2
    r = ofe.step(s, _frame(1), P, capacity=8)
    assert stand.calls == [("detect", 10, [0, 0, 0, 0]), ("track", 10, 11, 4)]
    assert s.xy[0].tolist() == [[10, 10], [60, 10], [10, 40], [60, 40]]
    assert s.ids[0].tolist() == [0, 1, 2, 3]
    assert s.xy[1].tolist() == [[3, 10], [53, 10], [3, 40]]
    assert s.ids[1].tolist() == [0, 1, 2]
    assert s.next_id == 4 and r["track"] == [None, None]
    assert r["occupancy"].tolist() == [0, 0, 0, 0]
    stand.calls.clear()
    # frame 2: camera 0 tracks move by (+1, +1) except (10, 40), which fails:
    # survivors (11, 11) id 0 -> cell 0, (61, 11) id 1 -> cell 1,
    # (61, 41) id 3 -> cell 3; occupancy [1, 1, 0, 1]; camera 1 tracks move by
    # (+2, 0) except (3, 40): survivors (5, 10) id 0, (55, 10) id 1. Only cell
    # 2 is free: new keypoint (10, 40), id 4, matched to (3, 40).
    r = ofe.step(s, _frame(2), P, capacity=8)
    assert stand.calls == [("track", 10, 20, 4), ("track", 11, 21, 3),
                           ("detect", 20, [1, 1, 0, 1]), ("track", 20, 21, 1)]
    assert r["occupancy"].tolist() == [1, 1, 0, 1]
    assert s.xy[0].tolist() == [[11, 11], [61, 11], [61, 41], [10, 40]]
    assert s.ids[0].tolist() == [0, 1, 3, 4]
    assert s.xy[1].tolist() == [[5, 10], [55, 10], [3, 40]]
    assert s.ids[1].tolist() == [0, 1, 4]
    assert s.next_id == 5
    assert s.pyr == [("pyr", 20), ("pyr", 21)]


def test_truncation_to_capacity(stand):
    # capacity 3: camera 0 keeps the first three new keypoints (raster order),
    # camera 1 the first three successful matches (ids 0, 1, 2); the id
    # counter still advances by the four detected
    s = ofe.StreamState()
    ofe.step(s, _frame(1), P, capacity=3)
    assert s.xy[0].tolist() == [[10, 10], [60, 10], [10, 40]]
    assert s.ids[0].tolist() == [0, 1, 2]
    assert s.ids[1].tolist() == [0, 1, 2]
    assert s.next_id == 4


def test_occupancy_rule():
    # floor(x / cw), floor(y / ch) over the full cells only; negative or
    # beyond-the-grid positions are not counted; counts saturate at 255
    xy = [(0.0, 0.0), (49.999, 29.999), (50.0, 0.0), (-0.5, 3.0), (3.0, -0.1),
          (100.0, 10.0), (99.9, 59.9), (10.0, 60.0)] + [(20.0, 40.0)] * 300
    occ = ofe.occupancy(np.array(xy, np.float32), W, H, CW, CH)
    assert occ.dtype == np.uint8
    assert occ.tolist() == [2, 1, 255, 1]
    # partial cells at the right and bottom edges belong to no cell
    occ2 = ofe.occupancy(np.array([(105.0, 5.0), (5.0, 65.0)], np.float32), 110, 70, CW, CH)
    assert occ2.tolist() == [0, 0, 0, 0]
