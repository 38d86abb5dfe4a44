"""GB300-native sixth-order compact Helmholtz solver: the helm6 C-ABI library (CUDA for
sm_103a, built in-tree by `build.build()`), its ctypes binding `helm6`, and the training
and evaluation of the learned second preconditioner stage (`learned`)."""
import os

_PKG = os.path.dirname(os.path.abspath(__file__))


def weights_path(name: str) -> str:
    """Path of a file under the package's weights/ folder (trained network parameters)."""
    return os.path.join(_PKG, "weights", name)
