// bitsliced_sbox.cuh -- GENERATED by gen_bitsliced_sbox.py; do not edit.
//
// The AES S-box without its constant 0x63 (FIPS-197 sec. 5.1.1: affine map of
// the inverse in GF(2^8)) as 129 gates (36 AND, 93 XOR), computed through the
// tower field GF(((2^2)^2)^2) with nu = 3, lambda = 11 (tower bit patterns).
// Each argument is one bit of the byte (b0 = least significant) for 32
// independent bytes, one per bit of the word; the outputs overwrite the
// inputs.  Checked on all 256 inputs by the generator.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gcmgpu {

__host__ __device__ __forceinline__ void sbox_bitsliced(uint32_t &b0, uint32_t &b1, uint32_t &b2,
                                                        uint32_t &b3, uint32_t &b4, uint32_t &b5,
                                                        uint32_t &b6, uint32_t &b7)
{
    const uint32_t t0 = b3 ^ b6;
    const uint32_t t1 = b5 ^ t0;
    const uint32_t t2 = b2 ^ b4;
    const uint32_t t3 = b1 ^ t1;
    const uint32_t t4 = b2 ^ b3;
    const uint32_t t5 = b7 ^ t2;
    const uint32_t t6 = b5 ^ b7;
    const uint32_t t7 = b2 ^ t0;
    const uint32_t t8 = t1 ^ t2;
    const uint32_t t9 = b1 ^ t0;
    const uint32_t t10 = t4 ^ t6;
    const uint32_t t11 = b0 ^ t7;
    const uint32_t t12 = b4 ^ b5;
    const uint32_t t13 = t2 ^ t3;
    const uint32_t t14 = t5 ^ t9;
    const uint32_t t15 = b1 ^ t10;
    const uint32_t t16 = b6 ^ t12;
    const uint32_t t17 = b4 ^ t9;
    const uint32_t t18 = b7 ^ t11;
    const uint32_t t19 = b7 ^ t3;
    const uint32_t t20 = b0 ^ b1;
    const uint32_t t21 = t20 ^ t5;
    const uint32_t t22 = b0 ^ t8;
    const uint32_t t23 = b0 ^ t3;
    const uint32_t t24 = b6 ^ b7;
    const uint32_t t25 = b3 ^ t5;
    const uint32_t t26 = t6 & t3;
    const uint32_t t27 = t13 & t17;
    const uint32_t t28 = t14 & t12;
    const uint32_t t29 = t10 & b7;
    const uint32_t t30 = b1 & t18;
    const uint32_t t31 = t15 & t11;
    const uint32_t t32 = t4 & t19;
    const uint32_t t33 = t8 & t21;
    const uint32_t t34 = t16 & t22;
    const uint32_t t35 = t30 ^ t33;
    const uint32_t t36 = t26 ^ t30;
    const uint32_t t37 = t23 ^ t28;
    const uint32_t t38 = t37 ^ t29;
    const uint32_t t39 = t38 ^ t36;
    const uint32_t t40 = t24 ^ t27;
    const uint32_t t41 = t40 ^ t31;
    const uint32_t t42 = t41 ^ t36;
    const uint32_t t43 = t25 ^ t29;
    const uint32_t t44 = t43 ^ t32;
    const uint32_t t45 = t44 ^ t35;
    const uint32_t t46 = t1 ^ t31;
    const uint32_t t47 = t46 ^ t34;
    const uint32_t t48 = t47 ^ t35;
    const uint32_t t49 = t45 ^ t48;
    const uint32_t t50 = t39 ^ t42;
    const uint32_t t51 = t45 ^ t50;
    const uint32_t t52 = t42 ^ t49;
    const uint32_t t53 = t42 ^ t48;
    const uint32_t t54 = t39 ^ t45;
    const uint32_t t55 = t49 ^ t50;
    const uint32_t t56 = t48 & t42;
    const uint32_t t57 = t45 & t39;
    const uint32_t t58 = t49 & t50;
    const uint32_t t59 = t51 ^ t56;
    const uint32_t t60 = t59 ^ t57;
    const uint32_t t61 = t52 ^ t57;
    const uint32_t t62 = t61 ^ t58;
    const uint32_t t63 = t60 ^ t62;
    const uint32_t t64 = t62 & t48;
    const uint32_t t65 = t63 & t45;
    const uint32_t t66 = t60 & t49;
    const uint32_t t67 = t62 & t53;
    const uint32_t t68 = t63 & t54;
    const uint32_t t69 = t60 & t55;
    const uint32_t t70 = t67 ^ t68;
    const uint32_t t71 = t68 ^ t69;
    const uint32_t t72 = t64 ^ t65;
    const uint32_t t73 = t65 ^ t66;
    const uint32_t t74 = t72 ^ t73;
    const uint32_t t75 = t70 ^ t71;
    const uint32_t t76 = t71 ^ t73;
    const uint32_t t77 = t70 ^ t72;
    const uint32_t t78 = t74 ^ t75;
    const uint32_t t79 = t73 & t6;
    const uint32_t t80 = t72 & t13;
    const uint32_t t81 = t74 & t14;
    const uint32_t t82 = t71 & t10;
    const uint32_t t83 = t70 & b1;
    const uint32_t t84 = t75 & t15;
    const uint32_t t85 = t76 & t4;
    const uint32_t t86 = t77 & t8;
    const uint32_t t87 = t78 & t16;
    const uint32_t t88 = t73 & t3;
    const uint32_t t89 = t72 & t17;
    const uint32_t t90 = t74 & t12;
    const uint32_t t91 = t71 & b7;
    const uint32_t t92 = t70 & t18;
    const uint32_t t93 = t75 & t11;
    const uint32_t t94 = t76 & t19;
    const uint32_t t95 = t77 & t21;
    const uint32_t t96 = t78 & t22;
    const uint32_t t97 = t81 ^ t84;
    const uint32_t t98 = t80 ^ t97;
    const uint32_t t99 = t90 ^ t92;
    const uint32_t t100 = t85 ^ t86;
    const uint32_t t101 = t93 ^ t94;
    const uint32_t t102 = t96 ^ t101;
    const uint32_t t103 = t98 ^ t100;
    const uint32_t t104 = t88 ^ t99;
    const uint32_t t105 = t83 ^ t91;
    const uint32_t t106 = t102 ^ t104;
    const uint32_t t107 = t103 ^ t105;
    const uint32_t t108 = t83 ^ t103;
    const uint32_t t109 = t108 ^ t106;
    const uint32_t t110 = t89 ^ t90;
    const uint32_t t111 = t110 ^ t91;
    const uint32_t t112 = t111 ^ t93;
    const uint32_t t113 = t89 ^ t95;
    const uint32_t t114 = t113 ^ t99;
    const uint32_t t115 = t114 ^ t101;
    const uint32_t t116 = t82 ^ t98;
    const uint32_t t117 = t116 ^ t106;
    const uint32_t t118 = t104 ^ t107;
    const uint32_t t119 = t102 ^ t107;
    const uint32_t t120 = t79 ^ t81;
    const uint32_t t121 = t120 ^ t100;
    const uint32_t t122 = t79 ^ t85;
    const uint32_t t123 = t122 ^ t87;
    const uint32_t t124 = t123 ^ t92;
    const uint32_t t125 = t124 ^ t94;
    const uint32_t t126 = t125 ^ t95;
    const uint32_t t127 = t126 ^ t97;
    const uint32_t t128 = t127 ^ t105;
    b0 = t109;
    b1 = t112;
    b2 = t115;
    b3 = t117;
    b4 = t118;
    b5 = t119;
    b6 = t121;
    b7 = t128;
}

}  // namespace gcmgpu
