// Compile-time dispatch over (dimension, order): D in {2, 3}, rho in 1..8.
#pragma once

#define FC2T2_CASE(DD, RR, BODY)                      \
    case (DD) * 16 + (RR): {                          \
        constexpr int D_ = (DD);                      \
        constexpr int R_ = (RR);                      \
        BODY;                                         \
    } break;

#define FC2T2_DISPATCH(dim, rho, BODY, ONBAD)         \
    switch ((dim) * 16 + (rho)) {                     \
        FC2T2_CASE(2, 1, BODY)                        \
        FC2T2_CASE(2, 2, BODY)                        \
        FC2T2_CASE(2, 3, BODY)                        \
        FC2T2_CASE(2, 4, BODY)                        \
        FC2T2_CASE(2, 5, BODY)                        \
        FC2T2_CASE(2, 6, BODY)                        \
        FC2T2_CASE(2, 7, BODY)                        \
        FC2T2_CASE(2, 8, BODY)                        \
        FC2T2_CASE(3, 1, BODY)                        \
        FC2T2_CASE(3, 2, BODY)                        \
        FC2T2_CASE(3, 3, BODY)                        \
        FC2T2_CASE(3, 4, BODY)                        \
        FC2T2_CASE(3, 5, BODY)                        \
        FC2T2_CASE(3, 6, BODY)                        \
        FC2T2_CASE(3, 7, BODY)                        \
        FC2T2_CASE(3, 8, BODY)                        \
        default: ONBAD;                               \
    }
