"""CPU oracle for the Gerchberg-Saxton phase-mask iteration (Kramer, Hagemann,
Luke, "Real-Time Phase Masks for Interactive Stimulation of Optogenetic
Neurons", Sec. II).

TEST INFRASTRUCTURE ONLY. The oracle is a plain, slow, FP64 restatement of the
method used to check the CUDA path. Only the test suite, the package smoke
check and the CPU-baseline leg of the benchmark may import it. The product path
never calls into this package, and this package never imports the product
package: the two share no code.

Parity status per function is listed in the header of ``gs_oracle``.
"""

from .gs_oracle import (  # noqa: F401
    TL_LIT,
    TD_DARK,
    fft2u,
    ifft2u,
    target_amplitude,
    proj_S,
    proj_M,
    gap_to_M,
    gap_to_S,
    gs_step,
    gs_run,
    consistent_target,
    physical_error,
    intensity_loss,
    intensity_loss_grad,
)
