"""Seeded synthetic inputs for the FIRM reconstruction path.

This module is shared by the CPU oracle, the CUDA path's tests and the
benchmark.  It holds only data synthesis -- phantoms, poses, shifts,
defocus-group parameters, analytic projections and noise -- and none of the
reconstruction method's arithmetic (no CTF, no Fourier slices, no spreading,
no kernel, no solver).  Images are therefore simulated without a CTF: the
method weights its samples by the CTF of the group an image belongs to, but the
synthetic pixels themselves are plain projections plus white noise.

Conventions (the paper's Section 3.1):
  * volume V is an N^3 array indexed [i3][i2][i1] (x = i1 fastest), with
    centred coordinate n_j = i_j - N/2;
  * a rotation R acts on the molecule, phi_R(x) = phi(R^{-1} x), so a blob
    at centre c appears in the projection image at (R c)_{1,2};
  * images are [m][i2][i1] with pixel centre x = (i1 - N/2, i2 - N/2);
  * a shift s moves the image content: I(x) = J(x - s);
  * the viewing direction of R is R^T e_3 (the third row of R).
"""
from .generate import (  # noqa: F401
    Blobs, phantom_blobs, blob_volume, haar_rotations, vmf_rotations,
    cap_rotations, mixed_rotations, rct_rotations, project_blobs, add_noise, uniform_shifts,
    ctf_group_table, config_inputs, CONFIGS, BATCH, batch_inputs,
)
