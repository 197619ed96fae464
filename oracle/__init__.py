"""FP64 CPU oracle for NURBS Splatting's forward and backward step.

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU
baseline leg import this package; the library never does, and this package
imports nothing from the library.  It is a plain, slow restatement of the
paper's definitions in PyTorch CPU float64 (autograd supplies the exact
derivative):

  nurbs     §3.1, Eq. 1-3: knot vectors from intervals, closed-curve wrapping,
            Cox-de Boor basis (full recursion, 0/0 := 0), C(u), C'(u), arc length
  sampling  §3.2, Eq. 4-5: contour counts and Gaussians with endpoint replicas;
            §3.3, Eq. 6-7 and Eq. S1-S3: boundary polyline, padded grid,
            unsigned distance, winding-number sign, sigmoid fill opacity
  raster    §3.4, Eq. 8-9: FP32 tile bin rule, (tile, layer, sample) order,
            brute-force and tiled front-to-back compositing
  pipeline  §3.5, Eq. 10: L2 loss, exact gradients, central differences

Parity status: every function is pinned by closed forms, identities or
brute force in tests/test_oracle_*.py.  The paper prints no numeric worked
example of an image or gradient, so no stored value comes from the paper.
"""
