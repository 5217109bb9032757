"""The smoke check the build entry point offers (GS(2), Bi-CGSTAB and
GMRES(20) on the 32 x 32 system against the oracle) runs green."""
import pytest

pytestmark = pytest.mark.gpu


def test_smoke_entry_point():
    import __graft_entry__

    __graft_entry__.smoke()
