"""Spline vs voxel reconstruction (Sec. 3, Fig. 4) on a head-like phantom:
50 CGLS iterations with quadratic B-splines and with voxels (degree 0, the
classic DDA) from the same exact, noisy cone-beam data.  The paper finds
the spline reconstruction better by 5.7 dB (28.02 vs 22.29 dB; mean gap
5.6 dB over its dataset); here the claim checked is the sign and a clear
margin of that gap, the numbers are printed."""
import pytest

pytestmark = pytest.mark.gpu


def test_spline_beats_voxel_reconstruction():
    from paper_2511_11078_gb300 import build as B
    from paper_2511_11078_gb300 import experiment as E
    from paper_2511_11078_gb300 import spl

    B.build()
    spl.lib()
    r = E.run(dims=(90, 90, 25), n_views=100, det=(90, 25), iters=50, degrees=(2, 0))
    print(r)
    # (the data residual is no criterion: the voxel model can fit the noisy
    # data more closely while reconstructing the function worse)
    assert r["degree_2"]["psnr_db"] > r["degree_0"]["psnr_db"] + 1.0
